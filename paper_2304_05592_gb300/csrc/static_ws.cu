// static_ws.cu -- wave_forward_static: forward modelling for callers that
// cannot allocate device memory themselves.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the time
// they need a forward model: a plugin whose host application has reserved all
// device memory up front, or a latency-critical loop that must not pay for an
// allocation and the device synchronisation it can bring.  wave_forward still
// needs a caller-supplied workspace; this entry point instead runs the same
// wave_forward path on a fixed scratch array that lives in the library itself.
//
// The array is a file-scope __device__ array of WAVE_STATIC_WORKSPACE_BYTES:
// every GPU on which the library's module is loaded holds it until the
// process exits.  In host code its name is only a host-side stand-in for the
// symbol, so each call looks up the device address on the current device with
// cudaGetSymbolAddress and passes it on as the workspace pointer.

#include "internal.h"

namespace {

__device__ __align__(256) unsigned char g_scratch[WAVE_STATIC_WORKSPACE_BYTES];

// Device address of g_scratch on the current device.  Looked up on every call
// (cudaGetSymbolAddress allocates nothing and is cheap once the module is
// loaded on the device) rather than cached, so the address stays right after a
// cudaDeviceReset or any other teardown of the device's context.
wave_status_t scratch_address(void** out)
{
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
        wave::note_cuda_error(cudaGetLastError());
        return WAVE_ERR_CUDA;
    }
    *out = p;
    return WAVE_OK;
}

}  // namespace

extern "C" wave_status_t wave_forward_static(const wave_grid_t* grid, const float* vel, int nshot, int nsrc,
                                             const float* src_xyz, const float* wavelet, int nrec,
                                             const float* rec_xyz, float* data, void* stream)
{
    size_t need = 0;
    wave_status_t st = wave_workspace_size(grid, 0, nshot, nsrc, src_xyz, nrec, rec_xyz, 0, 0, &need);
    if (st) return st;
    if (need > WAVE_STATIC_WORKSPACE_BYTES) return WAVE_ERR_WORKSPACE;
    void* scratch = nullptr;
    if ((st = scratch_address(&scratch))) return st;
    // wave_forward clears every part of the workspace that must start at zero
    // (both wavefields and the first row of receiver slots) before its time
    // loop, so what an earlier call left in the array does not leak into this one.
    st = wave_forward(grid, vel, nshot, nsrc, src_xyz, wavelet, nrec, rec_xyz, data, scratch,
                      WAVE_STATIC_WORKSPACE_BYTES, stream);
    if (st || nshot == 0) return st;
    // this entry point returns with its results complete: wait for the
    // stream and report the device-side errors of the call
    return wave_status_wait(scratch, stream, nullptr);
}
