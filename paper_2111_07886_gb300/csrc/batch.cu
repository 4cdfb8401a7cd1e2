// Batched subiterations of many independent scans (Table I run for each scan).
//
// Every tick advances each running scan of the batch by one subiteration.  The scans are grouped
// into classes that share one kernel instantiation (plane-group size G, arithmetic, candidate
// bins per view); for each class the per-scan argument structs of the tick are packed, with
// per-kernel virtual-block prefix tables, into one pinned buffer and copied to the device, and
// five persistent kernels (mu pass, forward + ratio, fused update, objective projection, RDP
// value) stride over the virtual blocks of all scans of the class.  A scan that skips a kernel
// this tick (no dynamic nu, no iteration end, finished) simply gets zero virtual blocks, so the
// launch sequence never changes and each class's tick is captured once as a CUDA graph and
// replayed.  The descriptor buffers are double-buffered: the host fills one while the previous
// tick's graph may still read the other.  Each scan keeps its own launch shapes and reduction
// scratch, so its results are bitwise the same alone or in any mix.
#include <string.h>

#include <vector>

#include "pet_common.cuh"
#include "profile.cuh"

namespace pet {

int sm_count();
void count_launches(long long n);

struct BatchClass {
    int G = 0, arith = 0, KC = 0;
    int cap = 0;                              // scan slots of this class
    std::vector<pet_state *> slot;            // nullptr = empty
    std::vector<bool> objective;              // per slot: plan objectives
    // descriptor buffers (pinned host + device), double-buffered
    size_t bytes = 0;
    char *host[2] = {nullptr, nullptr};
    char *dev[2] = {nullptr, nullptr};
    cudaEvent_t done[2] = {nullptr, nullptr};
    bool used[2] = {false, false};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaStream_t exec_stream[2] = {nullptr, nullptr};
    int next = 0;                             // descriptor buffer of the next tick

    // layout of one descriptor buffer
    size_t off_fwd = 0, off_upd = 0, off_mu = 0, off_objf = 0, off_objr = 0, off_pre = 0;
    void layout()
    {
        size_t o = 0;
        auto take = [&](size_t n) { size_t r = o; o = (o + n + 255) / 256 * 256; return r; };
        off_fwd = take(sizeof(FwdArgs) * cap);
        off_upd = take(sizeof(UpdateArgs) * cap);
        off_mu = take(sizeof(ImageArgs) * cap);
        off_objf = take(sizeof(FwdArgs) * cap);
        off_objr = take(sizeof(ImageArgs) * cap);
        off_pre = take(sizeof(int) * 5 * (cap + 1));
        bytes = o;
    }
};

static int kc_of(const pet_state *s) { return s->g->dev.K <= 2 ? 2 : 4; }

}  // namespace pet

struct pet_batch {
    int capacity = 0;
    int use_graph = 1;
    std::vector<pet::BatchClass *> classes;
    int grid = 0;
    cudaStream_t side = nullptr;            // mu passes run beside the forward projections
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

using namespace pet;

static void class_free(BatchClass *c)
{
    for (int b = 0; b < 2; ++b) {
        if (c->exec[b]) cudaGraphExecDestroy(c->exec[b]);
        if (c->done[b]) cudaEventDestroy(c->done[b]);
        cudaFreeHost(c->host[b]);
        cudaFree(c->dev[b]);
    }
    delete c;
}

extern "C" pet_status pet_batch_create(int capacity, int use_graph, pet_batch **out)
{
    if (!out || capacity < 1 || capacity > 4096)
        return fail(PET_ERR_INVALID, "pet_batch_create: need 1 <= capacity <= 4096");
    pet_batch *b = new pet_batch();
    b->capacity = capacity;
    b->use_graph = use_graph ? 1 : 0;
    b->grid = sm_count() * 4;
    cudaError_t e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        delete b;
        return cuda_fail(e, "pet_batch_create: side stream");
    }
    *out = b;
    return PET_OK;
}

extern "C" void pet_batch_destroy(pet_batch *b)
{
    if (!b) return;
    for (BatchClass *c : b->classes) {
        for (int k = 0; k < 2; ++k)
            if (c->done[k] && c->used[k]) cudaEventSynchronize(c->done[k]);
        class_free(c);
    }
    if (b->side) {
        cudaStreamSynchronize(b->side);
        cudaStreamDestroy(b->side);
        cudaEventDestroy(b->ev_fork);
        cudaEventDestroy(b->ev_join);
    }
    delete b;
}

static pet_status class_for(pet_batch *b, pet_state *s, BatchClass **out)
{
    const int G = s->g->dev.G, arith = s->arith, KC = kc_of(s);
    for (BatchClass *c : b->classes)
        if (c->G == G && c->arith == arith && c->KC == KC) { *out = c; return PET_OK; }
    BatchClass *c = new BatchClass();
    c->G = G;
    c->arith = arith;
    c->KC = KC;
    c->cap = b->capacity;
    c->slot.assign(c->cap, nullptr);
    c->objective.assign(c->cap, false);
    c->layout();
    for (int k = 0; k < 2; ++k) {
        cudaError_t e = cudaMallocHost((void **)&c->host[k], c->bytes);
        if (e == cudaSuccess) e = cudaMalloc((void **)&c->dev[k], c->bytes);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->done[k], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            class_free(c);
            return cuda_fail(e, "pet_batch: descriptor buffers");
        }
        memset(c->host[k], 0, c->bytes);
    }
    b->classes.push_back(c);
    *out = c;
    return PET_OK;
}

extern "C" pet_status pet_batch_add(pet_batch *b, pet_state *s, int with_objective, void *stream)
{
    if (!b || !s) return fail(PET_ERR_INVALID, "pet_batch_add: NULL argument");
    for (BatchClass *c : b->classes)
        for (pet_state *x : c->slot)
            if (x == s) return fail(PET_ERR_INVALID, "pet_batch_add: state already in the batch");
    BatchClass *c = nullptr;
    PET_TRY(class_for(b, s, &c));
    int free_slot = -1;
    for (int k = 0; k < c->cap; ++k)
        if (!c->slot[k]) { free_slot = k; break; }
    if (free_slot < 0) return fail(PET_ERR_OOM, "pet_batch_add: batch is full");
    if (with_objective && s->J == 0 && s->objcap > 0) {
        // Phi(f^0) before the first subiteration
        FwdArgs fa;
        ImageArgs ra;
        objective_args(s, s->objhist, &fa, &ra);
        cudaStream_t st = as_stream(stream);
        PET_TRY(launch_forward(fa, FWD_OBJECTIVE, s->arith, st));
        PET_TRY(launch_rdp_value(ra, s->arith, st));
    }
    c->slot[free_slot] = s;
    c->objective[free_slot] = with_objective != 0;
    return PET_OK;
}

extern "C" pet_status pet_batch_remove(pet_batch *b, pet_state *s)
{
    if (!b || !s) return fail(PET_ERR_INVALID, "pet_batch_remove: NULL argument");
    for (BatchClass *c : b->classes)
        for (int k = 0; k < c->cap; ++k)
            if (c->slot[k] == s) {
                // the slot's descriptors may still be read by an in-flight tick: wait for it
                for (int q = 0; q < 2; ++q)
                    if (c->used[q]) cudaEventSynchronize(c->done[q]);
                c->slot[k] = nullptr;
                return PET_OK;
            }
    return fail(PET_ERR_NOT_FOUND, "pet_batch_remove: state not in the batch");
}

static bool running(const pet_state *s)
{
    return s && s->J < s->prm.iterations * s->g->dev.M;
}

namespace pet {
// True when pet_batch_step would not wait for an earlier tick: every class with running scans
// has its next descriptor buffer free.
bool batch_can_step(const pet_batch *b)
{
    for (const BatchClass *c : b->classes) {
        bool any = false;
        for (const pet_state *s : c->slot) any = any || running(s);
        if (!any) continue;
        if (c->used[c->next] && cudaEventQuery(c->done[c->next]) == cudaErrorNotReady) return false;
    }
    return true;
}
}  // namespace pet

extern "C" int pet_batch_size(const pet_batch *b)
{
    if (!b) return -1;
    int n = 0;
    for (const BatchClass *c : b->classes)
        for (const pet_state *s : c->slot) n += running(s) ? 1 : 0;
    return n;
}

// The five batched launches of one class tick, reading descriptor buffer `dev`.
static pet_status class_launches(pet_batch *b, BatchClass *c, const char *dev, cudaStream_t st)
{
    const int cap = c->cap;
    const int *pre = reinterpret_cast<const int *>(dev + c->off_pre);
    // the shape structs only select the kernel instantiation (G, K); contents come from `dev`
    FwdArgs fs{};
    fs.g.G = c->G;
    fs.g.K = c->KC;
    UpdateArgs us{};
    us.g.G = c->G;
    us.g.K = c->KC;
    ImageArgs is{};
    is.g.G = c->G;
    is.g.K = c->KC;
    Batch bm{dev + c->off_mu, pre + 0 * (cap + 1), cap, b->grid};
    Batch bf{dev + c->off_fwd, pre + 1 * (cap + 1), cap, b->grid};
    Batch bu{dev + c->off_upd, pre + 2 * (cap + 1), cap, b->grid};
    Batch bo{dev + c->off_objf, pre + 3 * (cap + 1), cap, b->grid};
    Batch br{dev + c->off_objr, pre + 4 * (cap + 1), cap, b->grid};
    // mu passes on the side stream, joined before the update (a parallel branch in the graph)
    PET_CUDA(cudaEventRecord(b->ev_fork, st));
    PET_CUDA(cudaStreamWaitEvent(b->side, b->ev_fork, 0));
    PET_TRY(launch_mu_sum_batch(is, bm, c->arith, b->side));
    PET_CUDA(cudaEventRecord(b->ev_join, b->side));
    PET_TRY(launch_forward_batch(fs, bf, FWD_RATIO, c->arith, st));
    PET_CUDA(cudaStreamWaitEvent(st, b->ev_join, 0));
    PET_TRY(launch_update_batch(us, bu, c->arith, st));
    PET_TRY(launch_forward_batch(fs, bo, FWD_OBJECTIVE, c->arith, st));
    PET_TRY(launch_rdp_value_batch(is, br, c->arith, st));
    return PET_OK;
}

static pet_status class_tick(pet_batch *b, BatchClass *c, cudaStream_t st, int *running_after)
{
    const int cap = c->cap;
    const int buf = c->next;
    c->next ^= 1;
    if (c->used[buf]) PET_CUDA(cudaEventSynchronize(c->done[buf]));   // host may now overwrite it
    char *h = c->host[buf];
    FwdArgs *fwd = reinterpret_cast<FwdArgs *>(h + c->off_fwd);
    UpdateArgs *upd = reinterpret_cast<UpdateArgs *>(h + c->off_upd);
    ImageArgs *mu = reinterpret_cast<ImageArgs *>(h + c->off_mu);
    FwdArgs *objf = reinterpret_cast<FwdArgs *>(h + c->off_objf);
    ImageArgs *objr = reinterpret_cast<ImageArgs *>(h + c->off_objr);
    int *pre = reinterpret_cast<int *>(h + c->off_pre);
    int n[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k <= cap; ++k) {
        for (int t = 0; t < 5; ++t) pre[t * (cap + 1) + k] = n[t];
        if (k == cap) break;
        pet_state *s = c->slot[k];
        if (!running(s)) continue;
        SubiterPlan pl;
        plan_subiter(s, &pl, c->objective[k]);
        mu[k] = pl.mu_args;
        fwd[k] = pl.fwd;
        upd[k] = pl.upd;
        if (pl.mu) n[0] += pl.mu_args.nvb;
        n[1] += pl.fwd.nvb;
        n[2] += pl.upd.nvb;
        if (pl.objective) {
            objf[k] = pl.obj_fwd;
            objr[k] = pl.obj_rdp;
            n[3] += pl.obj_fwd.nvb;
            n[4] += pl.obj_rdp.nvb;
        }
        if (running(s)) ++*running_after;
    }
    // prefix tables must close at the totals; the loop above wrote pre[t][cap] = n[t]
    if (b->use_graph && st != nullptr) {       // the legacy default stream cannot be captured
        if (!c->exec[buf] || c->exec_stream[buf] != st) {
            if (c->exec[buf]) cudaGraphExecDestroy(c->exec[buf]);
            c->exec[buf] = nullptr;
            cudaGraph_t graph = nullptr;
            PET_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaMemcpyAsync(c->dev[buf], c->host[buf], c->bytes,
                                            cudaMemcpyHostToDevice, st);
            pet_status ls = e == cudaSuccess ? class_launches(b, c, c->dev[buf], st)
                                             : cuda_fail(e, "pet_batch: descriptor copy");
            cudaError_t ec = cudaStreamEndCapture(st, &graph);
            if (ls != PET_OK) { if (graph) cudaGraphDestroy(graph); return ls; }
            if (ec != cudaSuccess) return cuda_fail(ec, "pet_batch: end capture");
            e = cudaGraphInstantiate(&c->exec[buf], graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return cuda_fail(e, "pet_batch: graph instantiate");
            c->exec_stream[buf] = st;
        }
        PET_CUDA(cudaGraphLaunch(c->exec[buf], st));
        count_launches(5);
    } else {
        PET_CUDA(cudaMemcpyAsync(c->dev[buf], c->host[buf], c->bytes, cudaMemcpyHostToDevice, st));
        PET_TRY(class_launches(b, c, c->dev[buf], st));
    }
    PET_CUDA(cudaEventRecord(c->done[buf], st));
    c->used[buf] = true;
    return PET_OK;
}

extern "C" pet_status pet_batch_step(pet_batch *b, void *stream, int *running_after)
{
    if (!b) return fail(PET_ERR_INVALID, "pet_batch_step: NULL batch");
    cudaStream_t st = as_stream(stream);
    int run = 0;
    for (BatchClass *c : b->classes) {
        bool any = false;
        for (pet_state *s : c->slot) any = any || running(s);
        if (!any) continue;
        PET_TRY(class_tick(b, c, st, &run));
    }
    if (running_after) *running_after = run;
    return PET_OK;
}
