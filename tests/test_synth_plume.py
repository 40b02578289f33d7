"""The plume inputs: the patchy rock-physics relation is the identity without
CO2 and lowers the velocity monotonically with saturation, the generated
perturbations sit in the reservoir with 2-8 % largest drops, and the
generators are deterministic in their seed."""
import numpy as np

from paper_2304_05592_gb300 import synth


def test_patchy_identity_and_monotone():
    vp, rho = 3000.0, 310.0 * 3000.0 ** 0.25
    v0, r0 = synth.patchy_velocity(0.0, vp, rho, 0.25)
    assert abs(v0 - vp) < 1e-9 and abs(r0 - rho) < 1e-9
    sw = np.linspace(0, 1, 21)
    v, r = synth.patchy_velocity(sw, vp, rho, 0.25)
    assert np.all(np.diff(v) < 0)
    # density drops by phi sw (rho_co2 - rho_brine)
    np.testing.assert_allclose(r, rho + 0.25 * sw * (700.0 - 1000.0))


def test_plume_models_are_seeded_and_bounded():
    for s in range(20):
        b, dv = synth.plume_model(s, nx=160, nz=96)
        b2, dv2 = synth.plume_model(s, nx=160, nz=96)
        assert np.array_equal(b, b2) and np.array_equal(dv, dv2)
        drop = float(np.max(-dv / b))
        assert 0.02 - 1e-6 <= drop <= 0.08 + 1e-6
        assert np.all(dv <= 0)
        rows = np.nonzero(np.any(dv < -1e-3 * b, axis=1))[0]
        assert rows.min() > 0.4 * 96  # below the seal, not near the surface
