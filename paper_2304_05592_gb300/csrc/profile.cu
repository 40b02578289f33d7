// profile.cu -- launch counting and CUDA-event timing of the stencil kernels
// (sampled launches, or whole runs of consecutive launches).  Off by default;
// wave_profile_start/stop bracket a measured region.
#include <atomic>
#include <mutex>
#include <vector>

#include "internal.h"

namespace wave {
namespace {

struct Sample {
    cudaEvent_t start, stop;
    bool adjoint;
    long long launches;  // step launches the sample covers
};

std::atomic<long long> g_launches{0};
std::mutex g_mu;
bool g_on = false;
int g_every = 1;
long long g_seen = 0;
std::vector<Sample> g_samples;  // recorded during the current region
std::vector<cudaEvent_t> g_pool;
size_t g_pool_next = 0;
constexpr size_t kMaxSamples = 8192;
constexpr size_t kMaxRuns = 16384;
// Run mode (every = 0): one sample per run of consecutive step launches of one
// kind on one stream, so launches inside a run keep overlapping as they do
// unmeasured (programmatic dependent launch); a run ends when the kind or the
// stream changes or another library kernel is launched.
bool g_runs = false;
bool g_open = false;
cudaStream_t g_run_stream = nullptr;

cudaEvent_t take_event()
{
    if (g_pool_next == g_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        g_pool.push_back(e);
    }
    return g_pool[g_pool_next++];
}

thread_local cudaError_t t_last_error = cudaSuccess;

}  // namespace

void note_cuda_error(cudaError_t e)
{
    if (e != cudaSuccess) t_last_error = e;
}

// Ends the open run (caller holds g_mu): its stop event goes on its stream
// before whatever is queued next.
static void close_run()
{
    if (!g_open) return;
    cudaEventRecord(g_samples.back().stop, g_run_stream);
    g_open = false;
}

void count_launch(int n)
{
    g_launches.fetch_add(n, std::memory_order_relaxed);
    if (g_runs) {
        std::lock_guard<std::mutex> lock(g_mu);
        close_run();
    }
}

void count_step_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

bool profile_sample(bool adjoint, cudaStream_t s, cudaEvent_t* stop)
{
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_on) return false;
    if (g_runs) {
        if (g_open && g_samples.back().adjoint == adjoint && g_run_stream == s) {
            ++g_samples.back().launches;
            return false;
        }
        close_run();
        if (g_samples.size() >= kMaxRuns) return false;
        Sample smp;
        smp.start = take_event();
        smp.stop = take_event();
        smp.adjoint = adjoint;
        smp.launches = 1;
        if (!smp.start || !smp.stop) return false;
        cudaEventRecord(smp.start, s);
        g_samples.push_back(smp);
        g_open = true;
        g_run_stream = s;
        return false;
    }
    const bool take = (g_seen++ % g_every) == 0 && g_samples.size() < kMaxSamples;
    if (!take) return false;
    Sample smp;
    smp.start = take_event();
    smp.stop = take_event();
    smp.adjoint = adjoint;
    smp.launches = 1;
    if (!smp.start || !smp.stop) return false;
    cudaEventRecord(smp.start, s);
    g_samples.push_back(smp);
    *stop = smp.stop;
    return true;
}

void profile_close(cudaEvent_t stop, cudaStream_t s) { cudaEventRecord(stop, s); }

}  // namespace wave

using namespace wave;

extern "C" {

long long wave_launch_count(void) { return g_launches.load(); }

const char* wave_cuda_error_name(void) { return cudaGetErrorName(t_last_error); }

wave_status_t wave_profile_start(int every)
{
    if (every < 0) return WAVE_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    g_on = true;
    g_runs = every == 0;
    g_open = false;
    g_every = every > 0 ? every : 1;
    g_seen = 0;
    g_samples.clear();
    g_pool_next = 0;
    return WAVE_OK;
}

wave_status_t wave_profile_stop(double* fwd_ms, long long* fwd_n, double* adj_ms, long long* adj_n)
{
    std::lock_guard<std::mutex> lock(g_mu);
    close_run();
    g_on = false;
    g_runs = false;
    double f = 0.0, a = 0.0;
    long long nf = 0, na = 0;
    for (const Sample& smp : g_samples) {
        if (cudaEventSynchronize(smp.stop) != cudaSuccess) return WAVE_ERR_CUDA;
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, smp.start, smp.stop) != cudaSuccess) return WAVE_ERR_CUDA;
        if (smp.adjoint) {
            a += ms;
            na += smp.launches;
        } else {
            f += ms;
            nf += smp.launches;
        }
    }
    g_samples.clear();
    if (fwd_ms) *fwd_ms = f;
    if (fwd_n) *fwd_n = nf;
    if (adj_ms) *adj_ms = a;
    if (adj_n) *adj_n = na;
    return WAVE_OK;
}

}  // extern "C"
