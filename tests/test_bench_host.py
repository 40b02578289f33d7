"""Host-side bookkeeping of bench.py (no GPU): the algorithmic byte model of the
2D steps, and that the DRAM traffic recorded for the default kernels belongs to
the kernel source as it stands (a changed kernel must report no traffic until
it is measured again)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_step_bytes_model():
    n, s = 198912, 32
    # forward: u^k and u^{k-1} read, u^{k+1} written per shot; the model once per launch
    assert bench.step_bytes("fwd", n, s) == {"amortised": n * (12 * s + 4), "nominal": n * s * 16}
    # adjoint with imaging: three levels read and one written per shot; model and accumulator once
    assert bench.step_bytes("adj", n, s) == {"amortised": n * (16 * s + 12), "nominal": n * s * 28}
    # a BF16 store adds a 2-byte write per point to the forward and halves the stored level's read
    assert bench.step_bytes("fwd", n, 1, "bf16")["amortised"] == n * (14 + 4)
    assert bench.step_bytes("adj", n, 1, "bf16")["amortised"] == n * (14 + 12)


def test_recorded_traffic_matches_current_kernel_sources():
    h2d = bench.kernel_hash("k_step2d_sgt")
    h3d = bench.kernel_hash("k_step3d_tma")
    assert len(h2d) == 16 and len(h3d) == 16
    for which, v in ((0, 44), (1, 42)):  # the library's default 2D forward and adjoint
        func, name = bench.VARIANT_KERNEL[(which, v)][:2]
        assert bench.TRAFFIC.get((name, bench.kernel_hash(func))), name
    assert bench.TRAFFIC.get(("k_step3d_tma<8,76,8,fwd>", h3d))
    # traffic is keyed by the source: any other hash finds nothing
    assert bench.TRAFFIC.get((bench.VARIANT_KERNEL[(0, 44)][1], "0" * 16)) is None


def test_kernel_hash_is_deterministic_and_specific():
    assert bench.kernel_hash("k_step2d_sgt") == bench.kernel_hash("k_step2d_sgt")
    assert bench.kernel_hash("k_step2d_sgt") != bench.kernel_hash("k_step3d_tma")
    assert bench.kernel_hash("no_such_kernel") == ""
