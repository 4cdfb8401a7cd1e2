// Batched subiterations of many independent scans (Table I run for each scan).
//
// Every tick advances each running scan of the batch by one subiteration.  The scans are grouped
// into classes that share one kernel instantiation (plane-group size G, arithmetic, candidate
// bins per view, in-plane or 3-D prior, one line or sub-rays per bin); for each class the per-scan argument structs of the tick are packed, with
// per-kernel virtual-block prefix tables, into one pinned buffer and copied to the device, and
// five persistent kernels (mu pass, forward + ratio, fused update, objective projection, RDP
// value) stride over the virtual blocks of all scans of the class.  A scan that skips a kernel
// this tick (no dynamic nu, no iteration end, finished) simply gets zero virtual blocks, so the
// launch sequence never changes and each class's tick is captured once as a CUDA graph and
// replayed.  The descriptor buffers are double-buffered: the host fills one while the previous
// tick's graph may still read the other.  Each scan keeps its own launch shapes and reduction
// scratch, so its results are bitwise the same alone or in any mix.
//
// A class with a single running scan skips all of this and launches that scan's kernels directly
// (the launches of pet_subiter): at light load a served scan then runs as fast as alone.
// Descriptor buffers rotate over kBufs per class (the host may run that many ticks ahead of the
// GPU).  Before each replay the tick's kernel nodes are fitted to its work: a kernel that no scan
// needs this tick (the mu pass outside the dynamic-nu range, the objective between iteration ends)
// is disabled, and every other kernel's grid is cut to its virtual-block count when that is below
// the persistent grid, so a tick of a few small scans costs what their work costs.
#include <string.h>

#include <vector>

#include "pet_common.cuh"
#include "profile.cuh"

namespace pet {

int sm_count();
void count_launches(long long n);

constexpr int kBufs = 4;                      // descriptor buffers (ticks in flight) per class
constexpr int kKinds = 5;                     // mu pass, forward + ratio, update, objective x2

struct BatchClass {
    int G = 0, arith = 0, KC = 0;
    int z3 = 0;                               // 3-D prior (the generic update and mu kernels)
    int sub = 0;                              // sub-ray geometry (the sub-ray update kernel)
    int vox = 0;                              // detection factors: p per voxel (generic update)
    int tof = 0;                              // TOF geometries (the TOF projector and gather)
    int cap = 0;                              // scan slots of this class
    std::vector<pet_state *> slot;            // nullptr = empty
    std::vector<bool> objective;              // per slot: plan objectives
    // descriptor buffers (pinned host + device), rotating
    size_t bytes = 0;
    char *host[kBufs] = {};
    char *dev[kBufs] = {};
    cudaEvent_t done[kBufs] = {};
    bool used[kBufs] = {};
    cudaGraph_t graph[kBufs] = {};
    cudaGraphExec_t exec[kBufs] = {};
    cudaStream_t exec_stream[kBufs] = {};
    // the captured graph's kernel node of each kind, its captured parameters, and its state in
    // the instantiated graph (enabled, grid)
    cudaGraphNode_t knode[kBufs][kKinds] = {};
    cudaKernelNodeParams kparams[kBufs][kKinds] = {};
    int kgrid[kBufs][kKinds] = {};            // grid each kernel node is set to (0: disabled)
    int next = 0;                             // descriptor buffer of the next tick

    cudaGraphNode_t mnode[kBufs] = {};       // the captured descriptor copy
    int knsc[kBufs] = {};                     // scans each buffer's kernel nodes were set for

    // Layout of a descriptor buffer holding n scans: the five prefix tables first, then the
    // per-kind argument arrays.  The running scans of a tick are packed at positions 0..n-1,
    // so only the first `bytes` of the buffer travel to the device.
    struct Layout {
        size_t off_pre, off[kKinds], bytes;   // kinds: mu, forward, update, objective x2
        int n;
    };
    static Layout layout_for(int n)
    {
        Layout L{};
        size_t o = 0;
        auto take = [&](size_t b) { size_t r = o; o = (o + b + 255) / 256 * 256; return r; };
        L.n = n;
        L.off_pre = take(sizeof(int) * kKinds * (n + 1));
        L.off[0] = take(sizeof(ImageArgs) * n);
        L.off[1] = take(sizeof(FwdArgs) * n);
        L.off[2] = take(sizeof(UpdateArgs) * n);
        L.off[3] = take(sizeof(FwdArgs) * n);
        L.off[4] = take(sizeof(ImageArgs) * n);
        L.bytes = o;
        return L;
    }
    void layout() { bytes = layout_for(cap).bytes; }
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
    for (int b = 0; b < kBufs; ++b) {
        if (c->exec[b]) cudaGraphExecDestroy(c->exec[b]);
        if (c->graph[b]) cudaGraphDestroy(c->graph[b]);
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
        for (int k = 0; k < kBufs; ++k)
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
    const int G = s->g->dev.G, arith = s->arith, KC = kc_of(s), z3 = s->prm.rdp_3d;
    const int sub = s->g->dev.table, vox = s->attn ? 1 : 0, tof = s->g->dev.T > 1 ? 1 : 0;
    for (BatchClass *c : b->classes)
        if (c->G == G && c->arith == arith && c->KC == KC && c->z3 == z3 && c->sub == sub &&
            c->vox == vox && c->tof == tof) {
            *out = c;
            return PET_OK;
        }
    BatchClass *c = new BatchClass();
    c->G = G;
    c->arith = arith;
    c->KC = KC;
    c->z3 = z3;
    c->sub = sub;
    c->vox = vox;
    c->tof = tof;
    c->cap = b->capacity;
    c->slot.assign(c->cap, nullptr);
    c->objective.assign(c->cap, false);
    c->layout();
    for (int k = 0; k < kBufs; ++k) {
        cudaError_t e = host_malloc((void **)&c->host[k], c->bytes);
        if (e == cudaSuccess) e = dev_malloc((void **)&c->dev[k], c->bytes);
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
    if (s->prm.regularizer == PET_REG_TV)
        return fail(PET_ERR_INVALID, "pet_batch_add: the TV variant runs through pet_subiter / pet_reconstruct");
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
                for (int q = 0; q < kBufs; ++q)
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

// The Batch argument of kind t for descriptor layout L in device buffer `dev`.
static Batch batch_arg(const BatchClass::Layout &L, const char *dev, int t, int grid)
{
    const int *pre = reinterpret_cast<const int *>(dev + L.off_pre);
    return Batch{dev + L.off[t], pre + t * (L.n + 1), L.n, grid};
}

// The five batched launches of one class tick, reading descriptor buffer `dev` laid out as L.
// n: virtual blocks per kind, or nullptr (graph capture: every kernel at the full persistent
// grid; the replay fits them to each tick).  Without a graph a kernel with no work is skipped
// and the others get grids of min(virtual blocks, persistent grid).
static pet_status class_launches(pet_batch *b, BatchClass *c, const BatchClass::Layout &L,
                                 const char *dev, const int *n, cudaStream_t st, int *launched)
{
    // the shape structs only select the kernel instantiation (G, K); contents come from `dev`
    FwdArgs fs{};
    fs.g.G = c->G;
    fs.g.K = c->KC;
    fs.g.R = c->sub ? 2 : 1;                  // selects the sub-ray (table-driven) projector
    fs.g.table = c->sub;
    fs.g.T = c->tof ? 2 : 1;                  // selects the TOF projector (the count comes per scan)
    UpdateArgs us{};
    us.g.G = c->G;
    us.g.K = c->KC;
    us.g.R = c->sub ? 2 : 1;                  // selects the sub-ray kernel (the count comes per scan)
    us.g.table = c->sub;
    us.g.T = c->tof ? 2 : 1;                  // selects the TOF gather
    us.z3 = c->z3;
    us.vox = c->vox;
    ImageArgs is{};
    is.g.G = c->G;
    is.g.K = c->KC;
    is.z3 = c->z3;
    auto grid = [&](int t) { return n ? std::min(n[t], b->grid) : b->grid; };
    auto on = [&](int t) { return !n || n[t] > 0; };
    int cnt = 0;
    // mu passes on the side stream, joined before the update (a parallel branch in the graph)
    if (on(0)) {
        PET_CUDA(cudaEventRecord(b->ev_fork, st));
        PET_CUDA(cudaStreamWaitEvent(b->side, b->ev_fork, 0));
        PET_TRY(launch_mu_sum_batch(is, batch_arg(L, dev, 0, grid(0)), c->arith, b->side));
        PET_CUDA(cudaEventRecord(b->ev_join, b->side));
        ++cnt;
    }
    if (on(1)) { PET_TRY(launch_forward_batch(fs, batch_arg(L, dev, 1, grid(1)), FWD_RATIO, c->arith, st)); ++cnt; }
    if (on(0)) PET_CUDA(cudaStreamWaitEvent(st, b->ev_join, 0));
    if (on(2)) { PET_TRY(launch_update_batch(us, batch_arg(L, dev, 2, grid(2)), c->arith, st)); ++cnt; }
    if (on(3)) { PET_TRY(launch_forward_batch(fs, batch_arg(L, dev, 3, grid(3)), FWD_OBJECTIVE, c->arith, st)); ++cnt; }
    if (on(4)) { PET_TRY(launch_rdp_value_batch(is, batch_arg(L, dev, 4, grid(4)), c->arith, st)); ++cnt; }
    if (launched) *launched = cnt;
    return PET_OK;
}

// Finds the captured graph's descriptor copy and the kernel node of each kind (by the argument
// array its Batch argument points to, in the capture layout L) and keeps the kernel parameters
// for the per-tick updates.
static pet_status index_nodes(BatchClass *c, int buf, const BatchClass::Layout &L)
{
    size_t nn = 0;
    PET_CUDA(cudaGraphGetNodes(c->graph[buf], nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    PET_CUDA(cudaGraphGetNodes(c->graph[buf], nodes.data(), &nn));
    int found = 0;
    c->mnode[buf] = nullptr;
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType ty;
        PET_CUDA(cudaGraphNodeGetType(nd, &ty));
        if (ty == cudaGraphNodeTypeMemcpy) { c->mnode[buf] = nd; continue; }
        if (ty != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp;
        PET_CUDA(cudaGraphKernelNodeGetParams(nd, &kp));
        const Batch *bt = reinterpret_cast<const Batch *>(kp.kernelParams[1]);
        for (int t = 0; t < kKinds; ++t)
            if (bt->args == c->dev[buf] + L.off[t]) {
                c->knode[buf][t] = nd;
                c->kparams[buf][t] = kp;
                c->kgrid[buf][t] = (int)kp.gridDim.x;
                ++found;
            }
    }
    c->knsc[buf] = L.n;
    if (found != kKinds || !c->mnode[buf])
        return fail(PET_ERR_CUDA, "pet_batch: captured graph lacks a node");
    return PET_OK;
}

// Fits the instantiated graph of buffer `buf` to this tick: the descriptor copy to the packed
// layout L, kernels without work disabled, the others pointed at L and their grids cut to their
// virtual blocks.  Returns the kernels that will run.
static pet_status fit_graph(pet_batch *b, BatchClass *c, int buf, const BatchClass::Layout &L,
                            const int *n, int *launched)
{
    PET_CUDA(cudaGraphExecMemcpyNodeSetParams1D(c->exec[buf], c->mnode[buf], c->dev[buf],
                                                c->host[buf], L.bytes, cudaMemcpyHostToDevice));
    const bool relayout = c->knsc[buf] != L.n;
    int cnt = 0;
    for (int t = 0; t < kKinds; ++t) {
        const int want = n[t] > 0 ? std::min(n[t], b->grid) : 0;
        if (want == 0) {
            if (c->kgrid[buf][t] != 0)
                PET_CUDA(cudaGraphNodeSetEnabled(c->exec[buf], c->knode[buf][t], 0));
            c->kgrid[buf][t] = 0;
            continue;
        }
        ++cnt;
        if (want == c->kgrid[buf][t] && !relayout) continue;
        if (c->kgrid[buf][t] == 0) PET_CUDA(cudaGraphNodeSetEnabled(c->exec[buf], c->knode[buf][t], 1));
        cudaKernelNodeParams kp = c->kparams[buf][t];
        Batch arg = batch_arg(L, c->dev[buf], t, want);
        void *params[2] = {kp.kernelParams[0], &arg};
        kp.kernelParams = params;
        kp.gridDim.x = (unsigned)want;
        PET_CUDA(cudaGraphExecKernelNodeSetParams(c->exec[buf], c->knode[buf][t], &kp));
        c->kgrid[buf][t] = want;
    }
    // a disabled node keeps its old arguments; it is re-pointed when it is enabled again
    c->knsc[buf] = L.n;
    *launched = cnt;
    return PET_OK;
}

// A class with one running scan: the scan's own launches (the kernels and shapes of
// pet_subiter, so the same bits), without descriptor upload or graph replay.
static pet_status solo_tick(pet_batch *b, BatchClass *c, int k, cudaStream_t st)
{
    pet_state *s = c->slot[k];
    SubiterPlan pl;
    plan_subiter(s, &pl, c->objective[k]);
    if (pl.mu) {
        PET_CUDA(cudaEventRecord(b->ev_fork, st));
        PET_CUDA(cudaStreamWaitEvent(b->side, b->ev_fork, 0));
        PET_TRY(launch_mu_sum(pl.mu_args, pl.arith, b->side));
        PET_CUDA(cudaEventRecord(b->ev_join, b->side));
    }
    PET_TRY(launch_forward(pl.fwd, FWD_RATIO, pl.arith, st));
    if (pl.mu) PET_CUDA(cudaStreamWaitEvent(st, b->ev_join, 0));
    PET_TRY(launch_update(pl.upd, pl.arith, st));
    if (pl.objective) {
        PET_TRY(launch_forward(pl.obj_fwd, FWD_OBJECTIVE, pl.arith, st));
        PET_TRY(launch_rdp_value(pl.obj_rdp, pl.arith, st));
    }
    return PET_OK;
}

static pet_status class_tick(pet_batch *b, BatchClass *c, cudaStream_t st, int *running_after)
{
    const int cap = c->cap;
    const int buf = c->next;
    c->next = (c->next + 1) % kBufs;
    if (c->used[buf]) PET_CUDA(cudaEventSynchronize(c->done[buf]));   // host may now overwrite it
    int nrun = 0, solo = -1;
    for (int k = 0; k < cap; ++k)
        if (running(c->slot[k])) { ++nrun; solo = k; }
    if (nrun == 1) {
        PET_TRY(solo_tick(b, c, solo, st));
        if (running(c->slot[solo])) ++*running_after;
        PET_CUDA(cudaEventRecord(c->done[buf], st));
        c->used[buf] = true;
        return PET_OK;
    }
    // pack the running scans' arguments at positions 0..nrun-1 of the tick's layout
    const BatchClass::Layout L = BatchClass::layout_for(nrun);
    char *h = c->host[buf];
    ImageArgs *mu = reinterpret_cast<ImageArgs *>(h + L.off[0]);
    FwdArgs *fwd = reinterpret_cast<FwdArgs *>(h + L.off[1]);
    UpdateArgs *upd = reinterpret_cast<UpdateArgs *>(h + L.off[2]);
    FwdArgs *objf = reinterpret_cast<FwdArgs *>(h + L.off[3]);
    ImageArgs *objr = reinterpret_cast<ImageArgs *>(h + L.off[4]);
    int *pre = reinterpret_cast<int *>(h + L.off_pre);
    int n[kKinds] = {0, 0, 0, 0, 0};
    int pos = 0;
    for (int k = 0; k < cap; ++k) {
        pet_state *s = c->slot[k];
        if (!running(s)) continue;
        for (int t = 0; t < kKinds; ++t) pre[t * (nrun + 1) + pos] = n[t];
        SubiterPlan pl;
        plan_subiter(s, &pl, c->objective[k]);
        mu[pos] = pl.mu_args;
        fwd[pos] = pl.fwd;
        upd[pos] = pl.upd;
        if (pl.mu) n[0] += pl.mu_args.nvb;
        n[1] += pl.fwd.nvb;
        n[2] += pl.upd.nvb;
        if (pl.objective) {
            objf[pos] = pl.obj_fwd;
            objr[pos] = pl.obj_rdp;
            n[3] += pl.obj_fwd.nvb;
            n[4] += pl.obj_rdp.nvb;
        }
        if (running(s)) ++*running_after;
        ++pos;
    }
    for (int t = 0; t < kKinds; ++t) pre[t * (nrun + 1) + nrun] = n[t];   // tables close at the totals
    int launched = 0;
    if (b->use_graph && st != nullptr) {       // the legacy default stream cannot be captured
        if (!c->exec[buf] || c->exec_stream[buf] != st) {
            if (c->exec[buf]) cudaGraphExecDestroy(c->exec[buf]);
            if (c->graph[buf]) cudaGraphDestroy(c->graph[buf]);
            c->exec[buf] = nullptr;
            c->graph[buf] = nullptr;
            cudaGraph_t graph = nullptr;
            PET_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaMemcpyAsync(c->dev[buf], c->host[buf], L.bytes,
                                            cudaMemcpyHostToDevice, st);
            pet_status ls = e == cudaSuccess ? class_launches(b, c, L, c->dev[buf], nullptr, st, nullptr)
                                             : cuda_fail(e, "pet_batch: descriptor copy");
            cudaError_t ec = cudaStreamEndCapture(st, &graph);
            if (ls != PET_OK) { if (graph) cudaGraphDestroy(graph); return ls; }
            if (ec != cudaSuccess) return cuda_fail(ec, "pet_batch: end capture");
            c->graph[buf] = graph;                 // kept: its nodes address the per-tick updates
            PET_TRY(index_nodes(c, buf, L));
            e = cudaGraphInstantiate(&c->exec[buf], graph, 0);
            if (e != cudaSuccess) return cuda_fail(e, "pet_batch: graph instantiate");
            c->exec_stream[buf] = st;
        }
        PET_TRY(fit_graph(b, c, buf, L, n, &launched));
        PET_CUDA(cudaGraphLaunch(c->exec[buf], st));
        count_launches(launched);
    } else {
        PET_CUDA(cudaMemcpyAsync(c->dev[buf], c->host[buf], L.bytes, cudaMemcpyHostToDevice, st));
        PET_TRY(class_launches(b, c, L, c->dev[buf], n, st, &launched));
    }
    PET_CUDA(cudaEventRecord(c->done[buf], st));
    c->used[buf] = true;
    return PET_OK;
}

extern "C" pet_status pet_batch_step(pet_batch *b, void *stream, int *running_after)
{
    if (!b) return fail(PET_ERR_INVALID, "pet_batch_step: NULL batch");
    TraceRange tr("pet_batch_step");
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
