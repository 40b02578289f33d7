// extras.cu -- data conditioning and model-update kernels around the wave
// solver: the low-cut wavelet and band-limited noise of the paper's FWI
// experiment (section "Deep priors and normalizing flows": a Ricker wavelet
// stripped of its content under 4 Hz, plus additive coloured Gaussian noise
// whose band matches the clean data's), and the vector updates of an FWI
// iteration (v <- v + a d, then clamping to velocity bounds).
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "internal.h"

namespace wave {
namespace {

// Spectrum of a real series by direct DFT sums in double:
// X[k] = sum_n q[n] exp(-2 pi i k n / nt), k = 0 .. nt/2, times the high-pass
// gain H(f_k); one thread per frequency.
__global__ void k_lowcut_spectrum(const float* __restrict__ q, int nt, double df, double f_cut, double f_pass,
                                  double2* __restrict__ X)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > nt / 2) return;
    double re = 0.0, im = 0.0;
    for (int n = 0; n < nt; ++n) {
        const long long r = ((long long)k * n) % nt;  // exact argument reduction
        double s, c;
        sincospi(2.0 * (double)r / (double)nt, &s, &c);
        re += (double)q[n] * c;
        im -= (double)q[n] * s;
    }
    const double f = k * df;
    double h = 1.0;
    if (f < f_cut) h = 0.0;
    else if (f < f_pass) h = 0.5 * (1.0 - cospi((f - f_cut) / (f_pass - f_cut)));
    X[k] = make_double2(h * re, h * im);
}

// Inverse real DFT: out[n] = (1/nt) (X0 + 2 sum_{0<k<nt/2} Re(X_k e^{+i th}) + [nt even] X_{nt/2} (-1)^n).
__global__ void k_lowcut_inverse(const double2* __restrict__ X, int nt, float* __restrict__ out)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nt) return;
    const int nh = nt / 2;
    double acc = X[0].x;
    for (int k = 1; k <= nh; ++k) {
        const long long r = ((long long)k * n) % nt;
        double s, c;
        sincospi(2.0 * (double)r / (double)nt, &s, &c);
        const double term = X[k].x * c - X[k].y * s;
        acc += (nt % 2 == 0 && k == nh) ? term : 2.0 * term;
    }
    out[n] = (float)(acc / (double)nt);
}

// noise[s][t][r] = sum_k f[k] white[s][t - k + center][r] (zero outside [0, nt)).
__global__ void k_filter_traces(const float* __restrict__ white, int nshot, int nt, int nrec,
                                const float* __restrict__ f, int nf, int center, float* __restrict__ noise)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long total = (long long)nshot * nt * nrec;
    if (i >= total) return;
    const int r = (int)(i % nrec);
    const long long st = i / nrec;
    const int t = (int)(st % nt);
    const long long s = st / nt;
    const float* w = white + s * (long long)nt * nrec + r;
    float acc = 0.0f;
    for (int k = 0; k < nf; ++k) {
        const int tt = t - k + center;
        if (tt >= 0 && tt < nt) acc = fmaf(f[k], w[(long long)tt * nrec], acc);
    }
    noise[i] = acc;
}

constexpr int kNormBlocks = 256;

// Two squared norms in FP64, per-block partials (fixed order).
__global__ void __launch_bounds__(256) k_norm2_pair(long long n, const float* __restrict__ a,
                                                    const float* __restrict__ b, double* __restrict__ part)
{
    __shared__ double sa[256], sb[256];
    double x = 0.0, y = 0.0;
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += 256LL * gridDim.x) {
        x += (double)a[i] * (double)a[i];
        y += (double)b[i] * (double)b[i];
    }
    sa[threadIdx.x] = x;
    sb[threadIdx.x] = y;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sa[threadIdx.x] += sa[threadIdx.x + w];
            sb[threadIdx.x] += sb[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sa[0];
        part[2 * blockIdx.x + 1] = sb[0];
    }
}

// out = data + scale noise with scale = 10^(-snr/20) ||data|| / ||noise||.
__global__ void k_add_scaled(long long n, const float* __restrict__ data, const float* __restrict__ noise,
                             const double* __restrict__ part, double snr_db, float* __restrict__ out)
{
    __shared__ float scale;
    if (threadIdx.x == 0) {
        double nd = 0.0, nn = 0.0;
        for (int k = 0; k < kNormBlocks; ++k) {
            nd += part[2 * k];
            nn += part[2 * k + 1];
        }
        scale = nn > 0.0 ? (float)(pow(10.0, -snr_db / 20.0) * sqrt(nd / nn)) : 0.0f;
    }
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = fmaf(scale, noise[i], data[i]);
}

__global__ void k_axpy(long long n, float alpha, const float* __restrict__ x, float* __restrict__ y)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = fmaf(alpha, x[i], y[i]);
}

__global__ void k_axpby(long long n, float alpha, const float* __restrict__ x, float beta, float* __restrict__ y)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = fmaf(alpha, x[i], beta * y[i]);
}

__global__ void k_mul(long long n, const float* __restrict__ x, float* __restrict__ y)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = x[i] * y[i];
}

// Dot product in double: kDotBlocks partial sums over a fixed grid-stride
// split, then one block adds them in block order (same bits on every run).
constexpr int kDotBlocks = 256;

__global__ void k_dot_partial(long long n, const float* __restrict__ x, const float* __restrict__ y, double* part)
{
    __shared__ double sh[256];
    double acc = 0.0;
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += 256LL * kDotBlocks)
        acc = fma((double)x[i], (double)y[i], acc);
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_dot_final(const double* part, double* out)
{
    __shared__ double sh[kDotBlocks];
    sh[threadIdx.x] = part[threadIdx.x];
    __syncthreads();
    for (int w = kDotBlocks / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

__global__ void k_clamp(long long n, float lo, float hi, float* __restrict__ y)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = fminf(fmaxf(y[i], lo), hi);
}

wave_status_t launched()
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        note_cuda_error(e);
        return WAVE_ERR_CUDA;
    }
    return WAVE_OK;
}

unsigned blocks_for(long long n) { return (unsigned)std::min<long long>((n + 255) / 256, 8192); }

}  // namespace
}  // namespace wave

using namespace wave;

extern "C" {

size_t wave_lowcut_work_bytes(int nt) { return nt < 1 ? 0 : (size_t)(nt / 2 + 1) * sizeof(double2); }

wave_status_t wave_lowcut(const float* q, int nt, float dt, float f_cut, float f_pass, float* out, void* work,
                          void* stream)
{
    if (!q || !out || !work || nt < 1 || !(dt > 0.0f) || !(f_cut >= 0.0f) || !(f_pass > f_cut)) return WAVE_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    double2* X = static_cast<double2*>(work);
    const int nk = nt / 2 + 1;
    k_lowcut_spectrum<<<(nk + 127) / 128, 128, 0, s>>>(q, nt, 1.0 / ((double)nt * dt), f_cut, f_pass, X);
    k_lowcut_inverse<<<(nt + 127) / 128, 128, 0, s>>>(X, nt, out);
    return launched();
}

size_t wave_add_noise_work_bytes(int nshot, int nt, int nrec)
{
    if (nshot < 0 || nt < 1 || nrec < 0) return 0;
    const size_t n = (size_t)nshot * nt * nrec * sizeof(float);
    return ((n + 255) & ~(size_t)255) + 2 * kNormBlocks * sizeof(double);
}

wave_status_t wave_add_noise(const float* data, const float* white, int nshot, int nt, int nrec, const float* filt,
                             int nf, int center, double snr_db, float* out, void* work, void* stream)
{
    if (!data || !white || !filt || !out || !work || nshot < 0 || nt < 1 || nrec < 0 || nf < 1) return WAVE_ERR_ARG;
    const long long n = (long long)nshot * nt * nrec;
    if (n == 0) return WAVE_OK;
    cudaStream_t s = (cudaStream_t)stream;
    float* noise = static_cast<float*>(work);
    double* part = reinterpret_cast<double*>(static_cast<char*>(work) + ((n * sizeof(float) + 255) & ~(size_t)255));
    k_filter_traces<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(white, nshot, nt, nrec, filt, nf, center, noise);
    k_norm2_pair<<<kNormBlocks, 256, 0, s>>>(n, data, noise, part);
    k_add_scaled<<<blocks_for(n), 256, 0, s>>>(n, data, noise, part, snr_db, out);
    return launched();
}

wave_status_t wave_axpy(long long n, float alpha, const float* x, float* y, void* stream)
{
    if (n < 0 || !x || !y) return WAVE_ERR_ARG;
    if (n == 0) return WAVE_OK;
    k_axpy<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(n, alpha, x, y);
    return launched();
}

wave_status_t wave_axpby(long long n, float alpha, const float* x, float beta, float* y, void* stream)
{
    if (n < 0 || (n > 0 && (!x || !y))) return WAVE_ERR_ARG;
    if (n == 0) return WAVE_OK;
    count_launch();
    k_axpby<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(n, alpha, x, beta, y);
    return launched();
}

wave_status_t wave_mul(long long n, const float* x, float* y, void* stream)
{
    if (n < 0 || (n > 0 && (!x || !y))) return WAVE_ERR_ARG;
    if (n == 0) return WAVE_OK;
    count_launch();
    k_mul<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(n, x, y);
    return launched();
}

wave_status_t wave_dot(long long n, const float* x, const float* y, double* out, void* stream)
{
    static_assert(kDotBlocks == WAVE_DOT_PARTIALS, "the header's scratch count");
    if (n < 0 || !out || (n > 0 && (!x || !y))) return WAVE_ERR_ARG;  // n = 0: out[0] = 0
    cudaStream_t s = (cudaStream_t)stream;
    count_launch(2);
    k_dot_partial<<<kDotBlocks, 256, 0, s>>>(n, x, y, out + 1);
    k_dot_final<<<1, kDotBlocks, 0, s>>>(out + 1, out);
    return launched();
}

wave_status_t wave_clamp(long long n, float lo, float hi, float* y, void* stream)
{
    if (n < 0 || !y || !(lo <= hi)) return WAVE_ERR_ARG;
    if (n == 0) return WAVE_OK;
    k_clamp<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(n, lo, hi, y);
    return launched();
}

}  // extern "C"
