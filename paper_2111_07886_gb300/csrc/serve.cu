// Serving loop: continuous batching of reconstruction requests (no counterpart in the paper).
//
// submit() copies a request's data to host memory and queues it.  A preparer thread admits
// queued requests in arrival order while slots and the device-memory budget allow: it reuses or
// creates the geometry (cached by description; a scan whose sens differs reuses the tables with a
// scale factor), uploads counts, gamma and f^0 on its own stream and creates the scan's resident
// state.  A runner thread moves prepared states into batches and steps them continuously:
// requests that arrive while others are on the GPU join at the next step, and each step advances
// every running scan of a batch by one subiteration (graph-replayed batched kernels).  Scans are
// kept in one batch per kernel class (plane-group size, arithmetic, gather width), each on its
// own stream: the classes step independently and overlap on the device, so a short 2-D scan does
// not advance in lock-step with a clinical-size stacked one.  The class of the larger scans runs
// on the stream of higher priority, so a large scan advances at close to its own speed while the
// small ones fill the SMs it leaves.  A scan that has done T x M subiterations is read back (f^T
// and its objective history) and retired, freeing its memory and slot; poll() returns its result
// and latency (submit to result available).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "pet_common.cuh"

using namespace pet;

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t ticket = 0;
    pet_geometry_desc desc{};
    std::vector<int32_t> counts;
    std::vector<float> gamma;
    std::vector<float> img0;                 // empty: f^0 = 1
    std::vector<float> mult;                 // per-bin detection factors (empty: none)
    pet_params prm{};
    int with_objective = 0;
    double t_submit = 0, t_prep = 0, t_admit = 0, t_join = 0, t_final = 0, t_done = 0;
    pet_status status = PET_PENDING;
    std::string err;
    std::vector<float> img;                  // result f^T [P][N][N]
    std::vector<double> obj;                 // Phi(f^k), k = 0..T
    // runtime
    pet_geometry *geom = nullptr;            // cached, not owned
    pet_state *state = nullptr;
    size_t bytes = 0;                        // device bytes accounted for this request
    float *h_img = nullptr;                  // pinned readback
    double *h_obj = nullptr;                 // pinned readback (3 (T+1))
    size_t h_img_bytes = 0, h_obj_bytes = 0;
    float *d_img = nullptr;                  // device readback in the C-ABI layout
    cudaEvent_t ready = nullptr;
    bool retiring = false;
    struct SrvClass *cls = nullptr;          // batch the scan runs in
};

// One batch per kernel class, stepped on its own stream.
struct SrvClass {
    int G = 0, arith = 0, KC = 0;
    pet_batch *batch = nullptr;
    cudaStream_t st = nullptr;
    std::vector<Request *> running;
};

// desc without sens
typedef std::tuple<int, int, double, int, int, double, int, int, double, int, double, double> GeoKey;

static int tof_of(const pet_geometry_desc &d) { return d.tof_bins > 1 ? d.tof_bins : 1; }

GeoKey key_of(const pet_geometry_desc &d)
{
    const bool tof = d.tof_bins > 1;
    return GeoKey(d.n, d.nplanes, d.pixel_mm, d.nviews, d.nbins, d.bin_mm, d.nsubsets,
                  d.subrays > 1 ? d.subrays : 1, d.ring_mm > 0 ? d.ring_mm : 0.0, tof_of(d),
                  tof ? d.tof_bin_mm : 0.0, tof ? d.tof_fwhm_mm : 0.0);
}

size_t geometry_bytes(const pet_geometry_desc &d)
{
    return (size_t)d.nviews * (sizeof(ViewGeo) + sizeof(RayGeo) * d.nbins + sizeof(int)) +
           (size_t)d.n * d.n * 16 + reducer_bytes(4096, 4) + 1024 + bp_table_bytes_bound(d);
}

size_t request_bytes(const pet_geometry_desc &d, const pet_params &p, bool attn = false)
{
    const size_t G = d.nplanes == 1 ? 1 : 8;
    const size_t Pp = (d.nplanes + G - 1) / G * G;
    const size_t esz = p.precision == PET_PREC_FP64 ? 8 : 4;
    const size_t maxv = (d.nviews + d.nsubsets - 1) / d.nsubsets;
    const size_t SB = (size_t)d.nbins * tof_of(d);   // sinogram entries per view and plane
    return 3 * (size_t)d.n * d.n * Pp * esz + maxv * SB * Pp * esz +
           (size_t)d.nviews * SB * Pp * 8 + reducer_bytes(4096, 2) +
           (size_t)d.n * d.n * d.nplanes * 4 + (size_t)(p.iterations + 1) * 24 + 4096 +
           (attn ? (size_t)d.nviews * SB * Pp * 4 + (size_t)d.n * d.n * Pp * esz : 0);
}

}  // namespace

struct pet_server {
    size_t budget = 0;
    int max_slots = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request *> queue;
    std::deque<Request *> ready;
    std::vector<SrvClass *> classes;
    int nrunning = 0;
    int autotune = 0;                        // > 0: tune new geometries for that many concurrent scans
    long long tuned = 0;
    std::map<uint64_t, Request *> all;
    std::map<GeoKey, std::pair<pet_geometry *, size_t>> geoms;
    size_t used = 0;
    int preparing = 0;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::thread prep_thread, run_thread;
    cudaStream_t prep_stream = nullptr, run_stream = nullptr;
    // staging for uploads (preparer thread only)
    void *d_stage = nullptr;
    size_t stage_bytes = 0;
    size_t stage_accounted = 0;
    // pinned readback buffers, reused across requests (freeing pinned memory can stall the GPU)
    std::vector<std::pair<void *, size_t>> pinned_free;
    // statistics
    std::vector<double> latencies;
    double sum_queue = 0, sum_prep = 0, sum_run = 0, sum_readback = 0;
    long long submitted = 0, completed = 0, failed = 0;
    double t_first = -1, t_last = 0;
    std::string fatal;
};

static void finish(pet_server *sv, Request *r, pet_status st, const std::string &msg)
{
    r->status = st;
    r->err = msg;
    r->t_done = now_s();
    if (st != PET_OK) ++sv->failed;
}

static void *pinned_get(pet_server *sv, size_t bytes)
{
    std::lock_guard<std::mutex> lk(sv->mu);
    for (size_t k = 0; k < sv->pinned_free.size(); ++k)
        if (sv->pinned_free[k].second >= bytes) {
            void *p = sv->pinned_free[k].first;
            sv->pinned_free.erase(sv->pinned_free.begin() + k);
            return p;
        }
    return nullptr;
}

// call with sv->mu held
static void release_request(pet_server *sv, Request *r)
{
    cudaStream_t st = r->cls ? r->cls->st : sv->run_stream;
    if (r->state) { state_release(r->state, st); r->state = nullptr; }
    if (r->ready) { cudaEventDestroy(r->ready); r->ready = nullptr; }
    if (r->h_img) sv->pinned_free.push_back(std::make_pair((void *)r->h_img, r->h_img_bytes));
    if (r->h_obj) sv->pinned_free.push_back(std::make_pair((void *)r->h_obj, r->h_obj_bytes));
    if (r->d_img) cudaFreeAsync(r->d_img, st);
    r->h_img = nullptr;
    r->h_obj = nullptr;
    r->d_img = nullptr;
    sv->used -= std::min(sv->used, r->bytes);
    r->bytes = 0;
}

// ------------------------------------------------------------------------------------------
// preparer: admission by slots and device memory, geometry, upload, state creation
// ------------------------------------------------------------------------------------------
static pet_status prepare(pet_server *sv, Request *r)
{
    cudaStream_t st = sv->prep_stream;
    const pet_geometry_desc &d = r->desc;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->geoms.find(key_of(d));
        if (it != sv->geoms.end()) r->geom = it->second.first;
    }
    if (!r->geom) {
        pet_geometry_desc gdsc = d;
        pet_geometry *g = nullptr;
        PET_TRY(pet_geometry_create(&gdsc, st, &g));
        if (sv->autotune > 0) {
            pet_status ts = pet_autotune_batch(g, sv->autotune, st, nullptr);
            if (ts != PET_OK) { pet_geometry_destroy(g); return ts; }
        }
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->geoms[key_of(d)] = std::make_pair(g, geometry_bytes(d));
        if (sv->autotune > 0) ++sv->tuned;
        r->geom = g;
    }
    const size_t nsino = (size_t)d.nplanes * d.nviews * d.nbins * tof_of(d);
    const size_t nimg = (size_t)d.nplanes * d.n * d.n;
    const size_t sino_b = (nsino * 4 + 255) / 256 * 256;
    const size_t need = 3 * sino_b + nimg * 4 + 512;
    if (sv->stage_bytes < need) {
        cudaStreamSynchronize(st);
        cudaFree(sv->d_stage);
        sv->d_stage = nullptr;
        sv->stage_bytes = 0;
        PET_CUDA(dev_malloc(&sv->d_stage, need));
        sv->stage_bytes = need;
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->used += need - std::min(need, sv->stage_accounted);
        sv->stage_accounted = need;
    }
    char *base = reinterpret_cast<char *>(sv->d_stage);
    int32_t *dc = reinterpret_cast<int32_t *>(base);
    float *dg = reinterpret_cast<float *>(base + (nsino * 4 + 255) / 256 * 256);
    float *dm = r->mult.empty() ? nullptr : reinterpret_cast<float *>(base + 2 * sino_b);
    float *di = r->img0.empty() ? nullptr : reinterpret_cast<float *>(base + 3 * sino_b);
    PET_CUDA(cudaMemcpyAsync(dc, r->counts.data(), nsino * 4, cudaMemcpyHostToDevice, st));
    PET_CUDA(cudaMemcpyAsync(dg, r->gamma.data(), nsino * 4, cudaMemcpyHostToDevice, st));
    if (dm) PET_CUDA(cudaMemcpyAsync(dm, r->mult.data(), nsino * 4, cudaMemcpyHostToDevice, st));
    if (di) PET_CUDA(cudaMemcpyAsync(di, r->img0.data(), nimg * 4, cudaMemcpyHostToDevice, st));
    PET_TRY(state_create_loaded(r->geom, d.sens, dc, dg, dm, di, &r->prm, st, &r->state));
    r->h_img_bytes = nimg * 4;
    r->h_obj_bytes = (size_t)(r->prm.iterations + 1) * 3 * 8;
    r->h_img = reinterpret_cast<float *>(pinned_get(sv, r->h_img_bytes));
    if (!r->h_img) PET_CUDA(host_malloc((void **)&r->h_img, r->h_img_bytes));
    r->h_obj = reinterpret_cast<double *>(pinned_get(sv, r->h_obj_bytes));
    if (!r->h_obj) PET_CUDA(host_malloc((void **)&r->h_obj, r->h_obj_bytes));
    PET_CUDA(dev_malloc_async((void **)&r->d_img, nimg * 4, st));
    PET_CUDA(cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming));
    PET_CUDA(cudaStreamSynchronize(st));       // uploads done: the staging buffer is free again
    r->counts.clear();
    r->counts.shrink_to_fit();
    r->gamma.clear();
    r->gamma.shrink_to_fit();
    r->img0.clear();
    r->img0.shrink_to_fit();
    r->mult.clear();
    r->mult.shrink_to_fit();
    return PET_OK;
}

static void prep_loop(pet_server *sv)
{
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        sv->cv.wait(lk, [&] {
            if (sv->stop) return true;
            if (sv->queue.empty()) return false;
            const int slots = sv->nrunning + (int)sv->ready.size() + sv->preparing;
            if (slots >= sv->max_slots) return false;
            Request *h = sv->queue.front();
            const size_t need = request_bytes(h->desc, h->prm, !h->mult.empty()) +
                                (sv->geoms.count(key_of(h->desc)) ? 0 : geometry_bytes(h->desc));
            // admit when it fits, or when nothing else holds memory (it then fails or runs alone)
            return sv->used + need <= sv->budget || slots == 0;
        });
        if (sv->stop) return;
        Request *r = sv->queue.front();
        sv->queue.pop_front();
        const bool new_geo = sv->geoms.count(key_of(r->desc)) == 0;
        const size_t need = request_bytes(r->desc, r->prm, !r->mult.empty()) +
                            (new_geo ? geometry_bytes(r->desc) : 0);
        if (sv->used + need > sv->budget) {
            finish(sv, r, PET_ERR_OOM, "request needs more device memory than the server budget");
            sv->cv.notify_all();
            continue;
        }
        sv->used += need;
        r->bytes = request_bytes(r->desc, r->prm, !r->mult.empty());   // geometry bytes stay cached
        ++sv->preparing;
        r->t_prep = now_s();
        lk.unlock();
        pet_status st = prepare(sv, r);
        std::string msg = st == PET_OK ? "" : pet_last_error();
        lk.lock();
        --sv->preparing;
        if (st != PET_OK) {
            // the geometry's bytes were reserved with the request; they stay reserved only if
            // the geometry was created (it then stays in the cache)
            if (new_geo && sv->geoms.count(key_of(r->desc)) == 0)
                sv->used -= std::min(sv->used, geometry_bytes(r->desc));
            release_request(sv, r);
            finish(sv, r, st, msg);
        } else {
            r->t_admit = now_s();
            sv->ready.push_back(r);
        }
        sv->cv.notify_all();
    }
}

// ------------------------------------------------------------------------------------------
// runner: continuous batching
// ------------------------------------------------------------------------------------------
static pet_status start_readback(pet_server *sv, Request *r)
{
    (void)sv;
    cudaStream_t st = r->cls->st;
    const GeoDev &gd = r->geom->dev;
    const size_t nimg = (size_t)gd.P * gd.N * gd.N;
    PET_TRY(from_internal_image(gd, r->state->f[r->state->cur], r->d_img, r->state->arith == AR_FP64, 0, st));
    PET_CUDA(cudaMemcpyAsync(r->h_img, r->d_img, nimg * 4, cudaMemcpyDeviceToHost, st));
    PET_CUDA(cudaMemcpyAsync(r->h_obj, r->state->objhist,
                             (size_t)(r->prm.iterations + 1) * 3 * 8, cudaMemcpyDeviceToHost, st));
    PET_CUDA(cudaEventRecord(r->ready, st));
    r->retiring = true;
    r->t_final = now_s();
    return PET_OK;
}

static int kc_class(const pet_state *s) { return s->g->dev.K <= 2 ? 2 : 4; }

// The class batch of a state, created on first use (call with sv->mu held).
static pet_status class_of(pet_server *sv, const pet_state *s, SrvClass **out)
{
    const int G = s->g->dev.G, KC = kc_class(s);
    for (SrvClass *c : sv->classes)
        if (c->G == G && c->arith == s->arith && c->KC == KC) { *out = c; return PET_OK; }
    SrvClass *c = new SrvClass();
    c->G = G;
    c->arith = s->arith;
    c->KC = KC;
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    // stacked (8-plane) scans: highest priority; 2-D scans: lowest
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->st, cudaStreamNonBlocking, G > 1 ? hi : lo);
    if (e != cudaSuccess) { delete c; return cuda_fail(e, "pet_serve: class stream"); }
    pet_status r = pet_batch_create(sv->max_slots, 1, &c->batch);
    if (r != PET_OK) { cudaStreamDestroy(c->st); delete c; return r; }
    sv->classes.push_back(c);
    *out = c;
    return PET_OK;
}

static void fail_class(pet_server *sv, SrvClass *c, pet_status st, const std::string &msg)
{
    for (Request *r : c->running) {
        pet_batch_remove(c->batch, r->state);
        release_request(sv, r);
        finish(sv, r, st, msg);
    }
    sv->nrunning -= (int)c->running.size();
    c->running.clear();
}

static void run_loop(pet_server *sv)
{
    cudaSetDevice(sv->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            while (!sv->ready.empty()) {
                Request *r = sv->ready.front();
                sv->ready.pop_front();
                SrvClass *c = nullptr;
                pet_status st = class_of(sv, r->state, &c);
                if (st == PET_OK) {
                    r->cls = c;
                    st = pet_batch_add(c->batch, r->state, r->with_objective, c->st);
                }
                if (st != PET_OK) {
                    std::string msg = pet_last_error();
                    release_request(sv, r);
                    finish(sv, r, PET_ERR_CUDA, msg);
                    continue;
                }
                r->t_join = now_s();
                c->running.push_back(r);
                ++sv->nrunning;
            }
            if (sv->nrunning == 0) {
                if (sv->stop) return;
                sv->cv.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
        }
        // step every class whose previous ticks leave a descriptor buffer free
        bool stepped = false;
        for (SrvClass *c : sv->classes) {
            if (c->running.empty() || !batch_can_step(c->batch)) continue;
            int nrun = 0;
            pet_status st = pet_batch_step(c->batch, c->st, &nrun);
            stepped = true;
            if (st != PET_OK) {
                std::lock_guard<std::mutex> lk(sv->mu);
                sv->fatal = pet_last_error();
                fail_class(sv, c, st, sv->fatal);
                sv->cv.notify_all();
            }
        }
        std::vector<Request *> done;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            for (SrvClass *c : sv->classes)
                for (Request *r : c->running) {
                    const pet_state *s = r->state;
                    if (!r->retiring && s->J >= s->prm.iterations * s->g->dev.M) {
                        if (start_readback(sv, r) != PET_OK) {
                            r->retiring = true;
                            r->status = PET_ERR_CUDA;       // reported as failed when retired
                            r->err = pet_last_error();
                            r->t_final = now_s();
                            cudaEventRecord(r->ready, c->st);
                        }
                    }
                    if (r->retiring && cudaEventQuery(r->ready) != cudaErrorNotReady) done.push_back(r);
                }
        }
        for (Request *r : done) {
            pet_batch_remove(r->cls->batch, r->state);
            std::lock_guard<std::mutex> lk(sv->mu);
            std::vector<Request *> &run = r->cls->running;
            run.erase(std::find(run.begin(), run.end(), r));
            --sv->nrunning;
            if (r->status == PET_PENDING) {
                const GeoDev &gd = r->geom->dev;
                const size_t nimg = (size_t)gd.P * gd.N * gd.N;
                r->img.assign(r->h_img, r->h_img + nimg);
                const int T = r->prm.iterations;
                r->obj.resize(T + 1);
                for (int k = 0; k <= T; ++k)
                    r->obj[k] = r->with_objective ? r->h_obj[3 * k] - r->h_obj[3 * k + 1] +
                                                        r->prm.beta * r->h_obj[3 * k + 2]
                                                  : NAN;
                finish(sv, r, PET_OK, "");
                ++sv->completed;
                sv->latencies.push_back(r->t_done - r->t_submit);
                sv->sum_queue += r->t_prep - r->t_submit;
                sv->sum_prep += r->t_admit - r->t_prep;
                sv->sum_run += r->t_final - r->t_admit;
                sv->sum_readback += r->t_done - r->t_final;
                sv->t_last = r->t_done;
            }
            else {
                finish(sv, r, r->status, r->err);
            }
            release_request(sv, r);
            sv->cv.notify_all();
        }
        // nothing to enqueue: every class has its ticks in flight.  Poll again at once (a sleep
        // would oversleep by the timer slack and let the GPU run dry at light load).
        if (!stepped && done.empty()) std::this_thread::yield();
    }
}

extern "C" pet_status pet_serve_create(size_t hbm_budget_bytes, int max_slots, int device,
                                       pet_server **out)
{
    if (!out || max_slots < 1 || max_slots > 4096 || hbm_budget_bytes == 0)
        return fail(PET_ERR_INVALID, "pet_serve_create: need 1 <= max_slots <= 4096 and a budget > 0");
    *out = nullptr;
    PET_CUDA(cudaSetDevice(device));
    pet_server *sv = new pet_server();
    sv->budget = hbm_budget_bytes;
    sv->max_slots = max_slots;
    sv->device = device;
    cudaError_t e = cudaStreamCreateWithFlags(&sv->prep_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->run_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete sv;
        return cuda_fail(e, "pet_serve_create: streams");
    }
    sv->prep_thread = std::thread(prep_loop, sv);
    sv->run_thread = std::thread(run_loop, sv);
    *out = sv;
    return PET_OK;
}

extern "C" pet_status pet_serve_autotune(pet_server *sv, int concurrent)
{
    if (!sv || concurrent < 0 || concurrent > 4096)
        return fail(PET_ERR_INVALID, "pet_serve_autotune: need a server and 0 <= concurrent <= 4096");
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->autotune = concurrent;
    return PET_OK;
}

extern "C" pet_status pet_serve_submit(pet_server *sv, const pet_request *rq, uint64_t *ticket)
{
    if (!sv || !rq || !ticket || !rq->h_counts || !rq->h_gamma)
        return fail(PET_ERR_INVALID, "pet_serve_submit: NULL argument");
    const pet_geometry_desc &d = rq->geom;
    if (d.n < 1 || d.nplanes < 1 || d.nviews < 1 || d.nbins < 1 || d.nsubsets < 1 ||
        d.nsubsets > d.nviews || !(d.pixel_mm > 0) || !(d.bin_mm > 0) || !(d.sens > 0) ||
        d.subrays < 0 || d.subrays > 64)
        return fail(PET_ERR_INVALID, "pet_serve_submit: invalid geometry description");
    PET_TRY(check_params(&rq->params));
    if (rq->params.regularizer == PET_REG_TV)
        return fail(PET_ERR_INVALID, "pet_serve_submit: the TV variant runs through pet_reconstruct");
    const size_t nsino = (size_t)d.nplanes * d.nviews * d.nbins * tof_of(d);
    const size_t nimg = (size_t)d.nplanes * d.n * d.n;
    for (size_t k = 0; k < nsino; ++k)
        if (rq->h_counts[k] < 0 || !(rq->h_gamma[k] > 0.f) || !isfinite(rq->h_gamma[k]))
            return fail(PET_ERR_INVALID, "pet_serve_submit: need counts >= 0 and 0 < gamma < inf");
    if (rq->h_mult)
        for (size_t k = 0; k < nsino; ++k)
            if (!(rq->h_mult[k] >= 0.f) || !isfinite(rq->h_mult[k]))
                return fail(PET_ERR_INVALID, "pet_serve_submit: need finite detection factors >= 0");
    Request *r = new Request();
    r->desc = d;
    r->prm = rq->params;
    r->with_objective = rq->with_objective;
    r->counts.assign(rq->h_counts, rq->h_counts + nsino);
    r->gamma.assign(rq->h_gamma, rq->h_gamma + nsino);
    if (rq->h_img_init) r->img0.assign(rq->h_img_init, rq->h_img_init + nimg);
    if (rq->h_mult) r->mult.assign(rq->h_mult, rq->h_mult + nsino);
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) { delete r; return fail(PET_ERR_INVALID, "pet_serve_submit: server stopping"); }
    r->ticket = sv->next_ticket++;
    r->t_submit = now_s();
    if (sv->t_first < 0) sv->t_first = r->t_submit;
    ++sv->submitted;
    sv->all[r->ticket] = r;
    sv->queue.push_back(r);
    *ticket = r->ticket;
    sv->cv.notify_all();
    return PET_OK;
}

extern "C" pet_status pet_serve_poll(pet_server *sv, uint64_t ticket, float *h_img_out,
                                     double *h_obj_out, double *latency_s)
{
    if (!sv) return fail(PET_ERR_INVALID, "pet_serve_poll: NULL server");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return fail(PET_ERR_NOT_FOUND, "pet_serve_poll: unknown ticket");
    Request *r = it->second;
    if (r->status == PET_PENDING) return PET_PENDING;
    pet_status st = r->status;
    if (st == PET_OK) {
        if (h_img_out) memcpy(h_img_out, r->img.data(), r->img.size() * sizeof(float));
        if (h_obj_out) memcpy(h_obj_out, r->obj.data(), r->obj.size() * sizeof(double));
        if (latency_s) *latency_s = r->t_done - r->t_submit;
    } else {
        set_error(r->err);
    }
    sv->all.erase(it);
    delete r;
    return st;
}

extern "C" pet_status pet_serve_stats_get(pet_server *sv, pet_serve_stats *out)
{
    if (!sv || !out) return fail(PET_ERR_INVALID, "pet_serve_stats_get: NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = sv->submitted;
    out->completed = sv->completed;
    out->failed = sv->failed;
    out->running = sv->nrunning;
    out->queued = (long long)(sv->queue.size() + sv->ready.size() + sv->preparing);
    out->hbm_in_use = sv->used;
    std::vector<double> l = sv->latencies;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto pct = [&](double q) {
            const double pos = q * (l.size() - 1);
            const size_t a = (size_t)floor(pos), b = std::min(l.size() - 1, a + 1);
            return l[a] + (pos - a) * (l[b] - l[a]);
        };
        out->p50_s = pct(0.5);
        out->p99_s = pct(0.99);
        double m = 0;
        for (double x : l) m += x;
        out->mean_s = m / l.size();
        const double span = sv->t_last - sv->t_first;
        out->scans_per_s = span > 0 ? sv->completed / span : 0.0;
        out->mean_queue_s = sv->sum_queue / l.size();
        out->mean_prepare_s = sv->sum_prep / l.size();
        out->mean_run_s = sv->sum_run / l.size();
        out->mean_readback_s = sv->sum_readback / l.size();
    }
    out->tuned_geometries = sv->tuned;
    return PET_OK;
}

extern "C" void pet_serve_destroy(pet_server *sv)
{
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        // drop queued requests; running ones are finished by the runner before it exits
        for (Request *r : sv->queue) finish(sv, r, PET_ERR_INVALID, "server destroyed");
        sv->queue.clear();
    }
    sv->cv.notify_all();
    if (sv->prep_thread.joinable()) sv->prep_thread.join();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        for (Request *r : sv->ready) { release_request(sv, r); finish(sv, r, PET_ERR_INVALID, "server destroyed"); }
        sv->ready.clear();
    }
    sv->cv.notify_all();
    if (sv->run_thread.joinable()) sv->run_thread.join();
    cudaSetDevice(sv->device);
    cudaStreamSynchronize(sv->run_stream);
    for (SrvClass *c : sv->classes) {
        cudaStreamSynchronize(c->st);
        pet_batch_destroy(c->batch);
        c->batch = nullptr;
    }
    for (auto &kv : sv->all) {
        release_request(sv, kv.second);
        delete kv.second;
    }
    cudaStreamSynchronize(sv->run_stream);
    for (SrvClass *c : sv->classes) {
        cudaStreamSynchronize(c->st);
        cudaStreamDestroy(c->st);
        delete c;
    }
    sv->classes.clear();
    for (auto &kv : sv->pinned_free) cudaFreeHost(kv.first);
    for (auto &kv : sv->geoms) pet_geometry_destroy(kv.second.first);
    cudaFree(sv->d_stage);
    cudaStreamDestroy(sv->prep_stream);
    cudaStreamDestroy(sv->run_stream);
    delete sv;
}
