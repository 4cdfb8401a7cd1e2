// Launch accounting: a counter of every kernel this library launches, and optional CUDA-event
// timing per kernel kind (events recorded on the launching stream around each launch).
#include <mutex>
#include <vector>

#include "profile.cuh"

namespace pet {

static std::mutex g_mu;
static bool g_enabled = false;
static long long g_launches = 0;
struct Pair { cudaEvent_t a, b; };
static std::vector<Pair> g_pending[PET_K_COUNT];
static std::vector<Pair> g_pool;
static double g_ms[PET_K_COUNT];
static long long g_count[PET_K_COUNT];

static Pair get_pair()
{
    if (!g_pool.empty()) { Pair p = g_pool.back(); g_pool.pop_back(); return p; }
    Pair p{};
    cudaEventCreate(&p.a);
    cudaEventCreate(&p.b);
    return p;
}

LaunchScope::LaunchScope(int kind, cudaStream_t st) : kind_(kind), st_(st), active_(false)
{
    std::lock_guard<std::mutex> lk(g_mu);
    ++g_launches;
    if (!g_enabled) return;
    Pair p = get_pair();
    a_ = p.a;
    b_ = p.b;
    cudaEventRecord(a_, st_);
    active_ = true;
}

LaunchScope::~LaunchScope()
{
    if (!active_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEventRecord(b_, st_);
    g_pending[kind_].push_back(Pair{a_, b_});
}

bool profile_active()
{
    std::lock_guard<std::mutex> lk(g_mu);
    return g_enabled;
}

void count_launches(long long n)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_launches += n;
}

}  // namespace pet

using namespace pet;

extern "C" void pet_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_enabled = on != 0;
}

extern "C" long long pet_launch_count(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    return g_launches;
}

extern "C" pet_status pet_profile_read(int kind, double *total_ms, long long *launches)
{
    if (kind < 0 || kind >= PET_K_COUNT || !total_ms || !launches)
        return fail(PET_ERR_INVALID, "pet_profile_read: bad kind or NULL output");
    std::lock_guard<std::mutex> lk(g_mu);
    for (int k = 0; k < PET_K_COUNT; ++k) {
        for (Pair &p : g_pending[k]) {
            cudaError_t e = cudaEventSynchronize(p.b);
            if (e != cudaSuccess) return cuda_fail(e, "pet_profile_read");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, p.a, p.b);
            g_ms[k] += ms;
            g_count[k] += 1;
            g_pool.push_back(p);
        }
        g_pending[k].clear();
    }
    *total_ms = g_ms[kind];
    *launches = g_count[kind];
    return PET_OK;
}

extern "C" void pet_profile_reset(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    for (int k = 0; k < PET_K_COUNT; ++k) {
        for (Pair &p : g_pending[k]) {
            cudaEventSynchronize(p.b);
            g_pool.push_back(p);
        }
        g_pending[k].clear();
        g_ms[k] = 0.0;
        g_count[k] = 0;
    }
}
