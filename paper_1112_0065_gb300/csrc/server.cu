// Streaming server: per-beam gulps are admitted as they arrive, each runs on
// an execution slot (its own CUDA stream and buffers), and gulps of different
// beams overlap on the device -- continuous batching at gulp granularity.
//
// Per beam the device keeps two window buffers (ping-pong).  Gulp k's window
// holds the last L input samples before it (L = maxdelay rounded up to 64)
// followed by its G new samples; its dedispersion output, restricted to the
// G outputs that end in the new samples (absolute outputs
// [kG - maxdelay, (k+1)G - maxdelay), clipped at 0 for the first gulp), equals
// a one-shot dedispersion of the whole stream.  After its dedispersion the
// gulp copies its last L samples into the other window's head for gulp k+1,
// and records an event gulp k+1 waits for.
//
// A gulp runs in two stages on its slot's stream.  Stage A: upload the new
// samples, dedisperse, search.  A background worker sees stage A finish,
// reads the group count, and enqueues stage B: snippets, classifier scores
// (or the plain S/N cut when no classifier is loaded), and the copy of the
// candidates to pinned host memory; a host function stamps the completion
// time.  Slots are created lazily while free device memory stays above the
// configured reserve, up to max_slots; a submit with no free slot returns
// DD_ERR_BUSY.  Host waits are bounded (DD_ERR_TIMEOUT); nothing waits on the
// device.
//
// Triggered dumps: with trigger_snr > 0, stage A ends by selecting the first
// trigger_max candidates (in (d, t) order) with snr >= trigger_snr and copying
// the raw rows of their sweeps out of the window into slot memory; the window
// is reused only after that copy (an event per window), and stage B brings the
// dumps to pinned host memory for the callback.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "dd_internal.h"

namespace dd {
namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

__global__ void attach_scores_kernel(const dd_candidate *__restrict__ in, const float *__restrict__ logits, int n,
                                     int beam, dd_candidate *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    dd_candidate c = in[i];
    c.beam = beam;
    c.score = logits ? logits[i] : 0.0f;
    out[i] = c;
}

// First trigger_max candidates with snr >= thr, in list order: sel[0] = count,
// then (candidate index, first window sample of its dump) pairs.  The dump
// starts at the candidate's first input sample rounded down to 64 and holds
// ns samples (clamped to end inside the window).
__global__ void trigger_select_kernel(const dd_candidate *__restrict__ cands, const unsigned *__restrict__ ngroups,
                                      int max_cands, float thr, int trigger_max, long long first, long long win_nsamp,
                                      long long ns, long long *__restrict__ sel) {
    if (threadIdx.x != 0) return;
    const int n = min((int)*ngroups, max_cands);
    long long k = 0;
    for (int i = 0; i < n && k < trigger_max; ++i) {
        if (!(cands[i].snr >= thr)) continue;
        long long t0 = (first + cands[i].t) / 64 * 64;
        t0 = max(0LL, min(t0, win_nsamp - ns));
        sel[1 + 2 * k] = i;
        sel[2 + 2 * k] = t0;
        ++k;
    }
    sel[0] = k;
}

// Dump j, channel blockIdx.y: ld bytes of the window row from sample sel t0.
__global__ void trigger_copy_kernel(const uint8_t *__restrict__ win, long long win_ld, int nchan,
                                    const long long *__restrict__ sel, long long dump_ld,
                                    uint8_t *__restrict__ dump) {
    const int j = blockIdx.x, c = blockIdx.y;
    if (j >= sel[0]) return;
    const uint4 *src = reinterpret_cast<const uint4 *>(win + (long long)c * win_ld + sel[2 + 2 * j] / 4);
    uint4 *dst = reinterpret_cast<uint4 *>(dump + ((long long)j * nchan + c) * dump_ld);
    for (long long i = threadIdx.x; i < dump_ld / 16; i += blockDim.x) dst[i] = src[i];
}

struct Beam {
    Plan *plan = nullptr;
    size_t L = 0;           // history samples (multiple of 64, >= maxdelay)
    size_t ld = 0;          // bytes per channel row of a window
    uint8_t *win[2] = {nullptr, nullptr};
    int cur = 0;            // window the next gulp uses
    long long next_seq = 0;
    cudaEvent_t ready = nullptr;  // recorded by the last gulp after its history copy
    bool has_prev = false;
    uint32_t *tap = nullptr;      // optional copy of every gulp's dedispersed slice
    size_t tap_ld = 0, tap_cap = 0;
    cudaEvent_t win_free[2] = {nullptr, nullptr};  // the window's trigger dumps are copied out
    bool win_used[2] = {false, false};
    long long dump_ns = 0;        // samples per channel in a trigger dump
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_a = nullptr;
    uint32_t *out = nullptr;
    size_t ld_out = 0;
    dd_search *search = nullptr;
    dd_nn *nn = nullptr;
    uint16_t *snip = nullptr;
    float *logits = nullptr;
    dd_candidate *dcands = nullptr;
    dd_candidate *hcands = nullptr;  // pinned
    long long *d_sel = nullptr, *h_sel = nullptr;  // trigger selection (h_sel pinned)
    uint8_t *d_dump = nullptr, *h_dump = nullptr;  // trigger dumps (h_dump pinned)
    int ntrig = 0;
    int state = 0;                   // 0 free, 1 stage A, 2 stage B, 3 done (result not yet taken)
    dd_gulp_result res;
    std::atomic<int> b_done{0};
    std::atomic<double> t_done{0.0};
    int ngroups = 0;
};

void CUDART_CB host_done(void *p) {
    Slot *s = static_cast<Slot *>(p);
    s->t_done.store(now_s());
    s->b_done.store(1);
}

}  // namespace

struct Server {
    dd_server_config cfg;
    std::vector<Beam> beams;
    std::vector<Slot *> slots;
    size_t slot_bytes = 0;
    int nn_batch = 1024;
    std::vector<float> nn_params;
    bool have_nn = false;
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    dd_status worker_status = DD_OK;
    std::deque<Slot *> done_order;
    int device = 0;
    int maxdelay_max = 0;
    int trigger_max = 0;          // 0: triggers off
    size_t dump_bytes = 0;        // bytes of one dump (nchan_max rows)
    int nchan_max = 0;
    long long dump_ld_max = 0;
};

static void free_slot(Slot *s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    dd_search_destroy(s->search);
    dd_nn_destroy(s->nn);
    cudaFree(s->out);
    cudaFree(s->snip);
    cudaFree(s->logits);
    cudaFree(s->dcands);
    if (s->hcands) cudaFreeHost(s->hcands);
    cudaFree(s->d_sel);
    cudaFree(s->d_dump);
    if (s->h_sel) cudaFreeHost(s->h_sel);
    if (s->h_dump) cudaFreeHost(s->h_dump);
    if (s->ev_a) cudaEventDestroy(s->ev_a);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

static dd_status make_slot(Server *sv, Slot **out) {
    const dd_server_config &c = sv->cfg;
    Slot *s = new (std::nothrow) Slot();
    if (!s) return fail(DD_ERR_NOMEM, "host allocation failed");
    int ndm_max = 0, nchan_max = 0;
    size_t nout_max = 0;
    for (const Beam &b : sv->beams) {
        ndm_max = std::max(ndm_max, b.plan->ndm);
        nchan_max = std::max(nchan_max, b.plan->nchan);
        nout_max = std::max(nout_max, b.L + c.gulp_nsamp - (size_t)b.plan->maxdelay);
    }
    s->ld_out = (nout_max + 3) / 4 * 4;
    dd_search_config sc;
    memset(&sc, 0, sizeof(sc));
    sc.ndm_max = ndm_max;
    sc.n_max = c.gulp_nsamp;
    sc.nchan = nchan_max;
    sc.half_window = c.half_window;
    sc.nwidths = c.nwidths;
    for (int k = 0; k < c.nwidths; ++k) sc.widths[k] = c.widths[k];
    sc.thresh = c.thresh;
    sc.max_cands = c.max_cands;
    sc.full_map = 0;
    sc.baseline = 0;
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_a, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&s->out, (size_t)ndm_max * s->ld_out * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s->snip, (size_t)c.max_cands * 64 * 64 * 2);
    if (e == cudaSuccess) e = cudaMalloc(&s->logits, (size_t)c.max_cands * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s->dcands, (size_t)c.max_cands * sizeof(dd_candidate));
    if (e == cudaSuccess) e = cudaMallocHost(&s->hcands, (size_t)c.max_cands * sizeof(dd_candidate));
    if (e == cudaSuccess && sv->trigger_max > 0) {
        const size_t nsel = 1 + 2 * (size_t)sv->trigger_max;
        e = cudaMalloc(&s->d_sel, nsel * 8);
        if (e == cudaSuccess) e = cudaMallocHost(&s->h_sel, nsel * 8);
        if (e == cudaSuccess) e = cudaMalloc(&s->d_dump, (size_t)sv->trigger_max * sv->dump_bytes);
        if (e == cudaSuccess) e = cudaMallocHost(&s->h_dump, (size_t)sv->trigger_max * sv->dump_bytes);
    }
    if (e != cudaSuccess) {
        dd_status st = cuda_fail(e, "allocating a server slot");
        free_slot(s);
        return st;
    }
    dd_status st = dd_search_create(&s->search, &sc);
    if (st == DD_OK && sv->have_nn) {
        st = dd_nn_create(&s->nn, sv->nn_batch);
        if (st == DD_OK) st = dd_nn_set_params(s->nn, sv->nn_params.data());
    }
    if (st != DD_OK) {
        free_slot(s);
        return st;
    }
    *out = s;
    return DD_OK;
}

// Stage B of a slot whose stage A finished: snippets, scores, candidate copy.
static dd_status enqueue_stage_b(Server *sv, Slot *s) {
    const Beam &bm = sv->beams[s->res.beam];
    long long nhot = 0;
    int ng = 0;
    unsigned flags = 0;
    dd_status st = dd_search_result(s->search, &nhot, &ng, &flags, s->stream);
    if (st != DD_OK) return st;
    s->ngroups = ng;
    s->res.ngroups = ng;
    s->res.flags = flags;
    const int n = std::min(ng, sv->cfg.max_cands);
    const dd_candidate *dc = nullptr;
    st = dd_search_device_candidates(s->search, &dc);
    if (st != DD_OK) return st;
    if (n > 0 && sv->have_nn) {
        st = dd_search_snippets(s->search, n, s->snip, s->stream);
        for (int i = 0; i < n && st == DD_OK; i += sv->nn_batch) {
            const int k = std::min(sv->nn_batch, n - i);
            st = dd_nn_forward(s->nn, s->snip + (size_t)i * 64 * 64, k, s->logits + i, s->stream);
        }
        if (st != DD_OK) return st;
    }
    if (n > 0) {
        attach_scores_kernel<<<(n + 255) / 256, 256, 0, s->stream>>>(dc, sv->have_nn ? s->logits : nullptr, n,
                                                                       s->res.beam, s->dcands);
        DD_CUDA_TRY(cudaGetLastError());
        DD_CUDA_TRY(cudaMemcpyAsync(s->hcands, s->dcands, (size_t)n * sizeof(dd_candidate), cudaMemcpyDeviceToHost,
                                    s->stream));
    }
    s->ntrig = 0;
    if (sv->trigger_max > 0) {
        DD_CUDA_TRY(cudaMemcpyAsync(s->h_sel, s->d_sel, 8, cudaMemcpyDeviceToHost, s->stream));
        DD_CUDA_TRY(cudaStreamSynchronize(s->stream));
        s->ntrig = (int)s->h_sel[0];
        if (s->ntrig > 0) {
            const size_t one = (size_t)bm.plan->nchan * (size_t)(bm.dump_ns / 4);
            DD_CUDA_TRY(cudaMemcpyAsync(s->h_sel, s->d_sel, (1 + 2 * (size_t)s->ntrig) * 8, cudaMemcpyDeviceToHost,
                                        s->stream));
            DD_CUDA_TRY(cudaMemcpyAsync(s->h_dump, s->d_dump, (size_t)s->ntrig * one, cudaMemcpyDeviceToHost,
                                        s->stream));
        }
    }
    DD_CUDA_TRY(cudaLaunchHostFunc(s->stream, host_done, s));
    return DD_OK;
}

// Hand the gulp's dumps to the callback (worker thread; candidates and dumps are on the host).
static void fire_triggers(Server *sv, Slot *s) {
    if (!sv->cfg.trigger_fn || s->ntrig <= 0) return;
    const Beam &bm = sv->beams[s->res.beam];
    const size_t ld = (size_t)(bm.dump_ns / 4);
    const size_t one = (size_t)bm.plan->nchan * ld;
    const long long win0 = s->res.seq * (long long)sv->cfg.gulp_nsamp - (long long)bm.L;  // window sample 0
    for (int j = 0; j < s->ntrig; ++j) {
        const int i = (int)s->h_sel[1 + 2 * j];
        dd_trigger tr;
        memset(&tr, 0, sizeof(tr));
        tr.beam = s->res.beam;
        tr.nchan = bm.plan->nchan;
        tr.seq = s->res.seq;
        tr.cand = s->hcands[i];
        tr.cand.score = 0.0f;
        tr.t0 = win0 + s->h_sel[2 + 2 * j];
        tr.nsamp = bm.dump_ns;
        tr.ld = ld;
        sv->cfg.trigger_fn(sv->cfg.trigger_user, &tr, s->h_dump + (size_t)j * one);
    }
}

static void worker_loop(Server *sv) {
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (!sv->stop) {
        bool progressed = false;
        for (Slot *s : sv->slots) {
            if (s->state == 1) {
                const cudaError_t q = cudaEventQuery(s->ev_a);
                if (q == cudaSuccess) {
                    const dd_status st = enqueue_stage_b(sv, s);
                    if (st != DD_OK) {
                        sv->worker_status = st;
                        s->res.flags |= 0x80000000u;
                        s->t_done.store(now_s());
                        s->b_done.store(1);
                    }
                    s->state = 2;
                    progressed = true;
                } else if (q != cudaErrorNotReady) {
                    sv->worker_status = cuda_fail(q, "stage A of a gulp");
                    s->res.flags |= 0x80000000u;
                    s->t_done.store(now_s());
                    s->b_done.store(1);
                    s->state = 2;
                }
            }
            if (s->state == 2 && s->b_done.load()) {
                if (!(s->res.flags & 0x80000000u)) fire_triggers(sv, s);
                s->res.t_done = s->t_done.load();
                s->res.ncand = std::min(s->ngroups, sv->cfg.max_cands);
                s->state = 3;
                sv->done_order.push_back(s);
                progressed = true;
                sv->cv.notify_all();
            }
        }
        if (!progressed) sv->cv.wait_for(lk, std::chrono::microseconds(100));
    }
}

}  // namespace dd

using namespace dd;

extern "C" {

dd_status dd_server_create(dd_server **out, const dd_server_config *cfg, dd_plan *const *plans) {
    if (!out || !cfg || !plans) return fail(DD_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    const dd_server_config &c = *cfg;
    if (c.nbeams < 1 || c.nbeams > DD_BATCH_MAX_BEAMS || c.gulp_nsamp == 0 || c.gulp_nsamp % 64 != 0 ||
        c.max_slots < 1 || c.max_slots > 256 || c.max_cands < 1 || c.nn_batch < 0)
        return fail(DD_ERR_INVALID_ARG, "bad server configuration");
    Server *sv = new (std::nothrow) Server();
    if (!sv) return fail(DD_ERR_NOMEM, "host allocation failed");
    sv->cfg = c;
    sv->nn_batch = c.nn_batch > 0 ? c.nn_batch : 1024;
    sv->trigger_max = c.trigger_snr > 0.0f ? (c.trigger_max > 0 ? c.trigger_max : 4) : 0;
    if (sv->trigger_max > 64) {
        delete sv;
        return fail(DD_ERR_INVALID_ARG, "trigger_max must be 0..64");
    }
    cudaGetDevice(&sv->device);
    if (c.classifier_path && c.classifier_path[0]) {
        dd_nn *tmp = nullptr;
        dd_status st = dd_nn_create(&tmp, 1);
        if (st == DD_OK) st = dd_nn_load(tmp, c.classifier_path);
        if (st == DD_OK) {
            sv->nn_params.resize(DD_NN_PARAMS);
            st = dd_nn_get_params(tmp, sv->nn_params.data());
        }
        dd_nn_destroy(tmp);
        if (st != DD_OK) {
            delete sv;
            return st;
        }
        sv->have_nn = true;
    }
    sv->beams.resize(c.nbeams);
    for (int b = 0; b < c.nbeams; ++b) {
        Beam &bm = sv->beams[b];
        bm.plan = reinterpret_cast<Plan *>(plans[b]);
        if (!bm.plan) {
            dd_server_destroy(reinterpret_cast<dd_server *>(sv));
            return fail(DD_ERR_INVALID_ARG, "beam %d has no plan", b);
        }
        if ((size_t)bm.plan->maxdelay >= c.gulp_nsamp) {
            dd_server_destroy(reinterpret_cast<dd_server *>(sv));
            return fail(DD_ERR_INVALID_ARG, "gulp_nsamp must exceed every beam's maximum delay");
        }
        bm.L = ((size_t)bm.plan->maxdelay + 63) / 64 * 64;
        bm.ld = ((bm.L + c.gulp_nsamp) / 4 + 15) / 16 * 16;
        cudaError_t e = cudaMalloc(&bm.win[0], (size_t)bm.plan->nchan * bm.ld);
        if (e == cudaSuccess) e = cudaMalloc(&bm.win[1], (size_t)bm.plan->nchan * bm.ld);
        if (e == cudaSuccess) e = cudaMemset(bm.win[0], 0, (size_t)bm.plan->nchan * bm.ld);
        if (e == cudaSuccess) e = cudaMemset(bm.win[1], 0, (size_t)bm.plan->nchan * bm.ld);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bm.ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bm.win_free[0], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bm.win_free[1], cudaEventDisableTiming);
        bm.dump_ns = std::min((long long)(bm.L + c.gulp_nsamp), ((long long)bm.plan->maxdelay + 1024 + 63) / 64 * 64);
        sv->nchan_max = std::max(sv->nchan_max, bm.plan->nchan);
        sv->dump_ld_max = std::max(sv->dump_ld_max, bm.dump_ns / 4);
        if (e != cudaSuccess) {
            dd_status st = cuda_fail(e, "allocating beam windows");
            dd_server_destroy(reinterpret_cast<dd_server *>(sv));
            return st;
        }
    }
    // bytes one slot needs, for admission (estimated from its allocations)
    size_t ndm = 0, nout = 0;
    for (const Beam &b : sv->beams) {
        ndm = std::max(ndm, (size_t)b.plan->ndm);
        nout = std::max(nout, b.L + c.gulp_nsamp);
    }
    sv->dump_bytes = (size_t)sv->nchan_max * (size_t)sv->dump_ld_max;
    sv->slot_bytes = ndm * nout * 4 + ndm * c.gulp_nsamp * 14 + (size_t)c.max_cands * (8192 + 64) +
                     ((size_t)1 << 27) + (size_t)sv->trigger_max * sv->dump_bytes;
    sv->worker = std::thread(worker_loop, sv);
    *out = reinterpret_cast<dd_server *>(sv);
    return DD_OK;
}

dd_status dd_server_set_tap(dd_server *server, int beam, uint32_t *d_dst, size_t ld_dst, size_t capacity) {
    Server *sv = reinterpret_cast<Server *>(server);
    if (!sv || beam < 0 || beam >= (int)sv->beams.size()) return fail(DD_ERR_INVALID_ARG, "bad server or beam");
    std::lock_guard<std::mutex> lk(sv->mu);
    Beam &b = sv->beams[beam];
    b.tap = d_dst;
    b.tap_ld = ld_dst;
    b.tap_cap = capacity;
    return DD_OK;
}

dd_status dd_server_submit(dd_server *server, int beam, const uint8_t *h_new, size_t h_pitch, long long *seq) {
    Server *sv = reinterpret_cast<Server *>(server);
    if (!sv || !h_new) return fail(DD_ERR_INVALID_ARG, "NULL server or gulp");
    if (beam < 0 || beam >= (int)sv->beams.size()) return fail(DD_ERR_INVALID_ARG, "beam %d out of range", beam);
    const size_t G = sv->cfg.gulp_nsamp;
    if (h_pitch < G / 4) return fail(DD_ERR_INVALID_ARG, "host pitch %zu below the gulp's %zu bytes", h_pitch, G / 4);
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->worker_status != DD_OK) return sv->worker_status;
    // admission: a free slot, or a new one while device memory allows
    Slot *s = nullptr;
    for (Slot *x : sv->slots)
        if (x->state == 0) {
            s = x;
            break;
        }
    if (!s) {
        if ((int)sv->slots.size() >= sv->cfg.max_slots) return fail(DD_ERR_BUSY, "all %d slots in flight", sv->cfg.max_slots);
        size_t fr = 0, tot = 0;
        DD_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
        if (fr < sv->cfg.hbm_reserve_bytes + sv->slot_bytes)
            return fail(DD_ERR_BUSY, "free device memory %zu below reserve + slot (%zu)", fr,
                        sv->cfg.hbm_reserve_bytes + sv->slot_bytes);
        dd_status st = make_slot(sv, &s);
        if (st == DD_ERR_NOMEM) return fail(DD_ERR_BUSY, "device memory ran out creating a slot");
        if (st != DD_OK) return st;
        sv->slots.push_back(s);
    }
    Beam &bm = sv->beams[beam];
    Plan *p = bm.plan;
    const int w = bm.cur;
    const long long k = bm.next_seq;
    cudaStream_t st = s->stream;
    s->res = dd_gulp_result();
    s->res.beam = beam;
    s->res.seq = k;
    s->res.t_submit = now_s();
    s->b_done.store(0);
    s->ngroups = 0;
    // stage A
    if (bm.has_prev) DD_CUDA_TRY(cudaStreamWaitEvent(st, bm.ready, 0));
    if (sv->trigger_max > 0 && bm.win_used[w]) DD_CUDA_TRY(cudaStreamWaitEvent(st, bm.win_free[w], 0));
    DD_CUDA_TRY(cudaMemcpy2DAsync(bm.win[w] + bm.L / 4, bm.ld, h_new, h_pitch, G / 4, p->nchan, cudaMemcpyHostToDevice,
                                  st));
    const size_t nsamp = bm.L + G;
    dd_status ds = dd_execute(reinterpret_cast<const dd_plan *>(p), bm.win[w], bm.ld, nsamp, s->out, s->ld_out, st);
    if (ds != DD_OK) return ds;
    // the history copy overwrites the start of the other window, which the previous gulp's trigger
    // dumps may still be reading (a dump can start inside its history)
    if (sv->trigger_max > 0 && bm.win_used[w ^ 1]) DD_CUDA_TRY(cudaStreamWaitEvent(st, bm.win_free[w ^ 1], 0));
    DD_CUDA_TRY(cudaMemcpy2DAsync(bm.win[w ^ 1], bm.ld, bm.win[w] + G / 4, bm.ld, bm.L / 4, p->nchan,
                                  cudaMemcpyDeviceToDevice, st));
    DD_CUDA_TRY(cudaEventRecord(bm.ready, st));
    // outputs ending in the new samples: window outputs [L - maxdelay, L - maxdelay + G); the first
    // gulp has no history, so its slice starts at window output L (absolute output 0)
    const size_t first = k == 0 ? bm.L : bm.L - (size_t)p->maxdelay;
    const size_t n = bm.L - (size_t)p->maxdelay + G - first;
    const long long t_abs = k == 0 ? 0 : k * (long long)G - p->maxdelay;
    s->res.t0 = t_abs;
    s->res.nout = (long long)n;
    if (bm.tap && (size_t)t_abs + n <= bm.tap_cap)
        DD_CUDA_TRY(cudaMemcpy2DAsync(bm.tap + t_abs, bm.tap_ld * 4, s->out + first, s->ld_out * 4, n * 4, p->ndm,
                                      cudaMemcpyDeviceToDevice, st));
    ds = dd_search_run(s->search, s->out + first, s->ld_out, p->ndm, n, beam, st);
    if (ds != DD_OK) return ds;
    if (sv->trigger_max > 0) {
        const dd_candidate *dc = nullptr;
        ds = dd_search_device_candidates(s->search, &dc);
        if (ds != DD_OK) return ds;
        trigger_select_kernel<<<1, 32, 0, st>>>(dc, search_dev_ngroups(s->search), sv->cfg.max_cands,
                                                sv->cfg.trigger_snr, sv->trigger_max, (long long)first,
                                                (long long)nsamp, bm.dump_ns, s->d_sel);
        trigger_copy_kernel<<<dim3((unsigned)sv->trigger_max, (unsigned)p->nchan), 128, 0, st>>>(
            bm.win[w], (long long)bm.ld, p->nchan, s->d_sel, bm.dump_ns / 4, s->d_dump);
        DD_CUDA_TRY(cudaGetLastError());
        DD_CUDA_TRY(cudaEventRecord(bm.win_free[w], st));
        bm.win_used[w] = true;
    }
    DD_CUDA_TRY(cudaEventRecord(s->ev_a, st));
    bm.cur = w ^ 1;
    bm.has_prev = true;
    bm.next_seq = k + 1;
    s->state = 1;
    if (seq) *seq = k;
    sv->cv.notify_all();
    return DD_OK;
}

dd_status dd_server_poll(dd_server *server, dd_gulp_result *results, int max_results, int *nresults,
                         dd_candidate *cands, int max_cands_total, int *ncands, double wait_s) {
    Server *sv = reinterpret_cast<Server *>(server);
    if (!sv || !nresults) return fail(DD_ERR_INVALID_ARG, "NULL argument");
    std::unique_lock<std::mutex> lk(sv->mu);
    if (wait_s > 0 && sv->done_order.empty())
        sv->cv.wait_for(lk, std::chrono::duration<double>(wait_s), [&] { return !sv->done_order.empty(); });
    int nr = 0, nc = 0;
    while (!sv->done_order.empty() && nr < max_results) {
        Slot *s = sv->done_order.front();
        const int k = s->res.ncand;
        if (cands && nc + k > max_cands_total && nr > 0) break;
        dd_gulp_result r = s->res;
        r.cand_offset = nc;
        if (cands) {
            const int take = std::min(k, max_cands_total - nc);
            memcpy(cands + nc, s->hcands, (size_t)std::max(take, 0) * sizeof(dd_candidate));
            r.ncand = std::max(take, 0);
            nc += r.ncand;
        }
        if (results) results[nr] = r;
        ++nr;
        s->state = 0;
        sv->done_order.pop_front();
    }
    *nresults = nr;
    if (ncands) *ncands = nc;
    return sv->worker_status;
}

dd_status dd_server_drain(dd_server *server, double timeout_s) {
    Server *sv = reinterpret_cast<Server *>(server);
    if (!sv) return fail(DD_ERR_INVALID_ARG, "NULL server");
    std::unique_lock<std::mutex> lk(sv->mu);
    const bool ok = sv->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] {
        for (Slot *s : sv->slots)
            if (s->state == 1 || s->state == 2) return false;
        return true;
    });
    if (!ok) return fail(DD_ERR_TIMEOUT, "gulps still in flight after %.1f s", timeout_s);
    return sv->worker_status;
}

dd_status dd_server_info(const dd_server *server, int *nslots, int *in_flight, size_t *slot_bytes) {
    const Server *sv = reinterpret_cast<const Server *>(server);
    if (!sv) return fail(DD_ERR_INVALID_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(const_cast<Server *>(sv)->mu);
    int f = 0;
    for (Slot *s : sv->slots) f += (s->state == 1 || s->state == 2);
    if (nslots) *nslots = (int)sv->slots.size();
    if (in_flight) *in_flight = f;
    if (slot_bytes) *slot_bytes = sv->slot_bytes;
    return DD_OK;
}

void dd_server_destroy(dd_server *server) {
    Server *sv = reinterpret_cast<Server *>(server);
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->cv.notify_all();
    }
    if (sv->worker.joinable()) sv->worker.join();
    for (Slot *s : sv->slots) free_slot(s);
    for (Beam &b : sv->beams) {
        cudaFree(b.win[0]);
        cudaFree(b.win[1]);
        if (b.ready) cudaEventDestroy(b.ready);
        if (b.win_free[0]) cudaEventDestroy(b.win_free[0]);
        if (b.win_free[1]) cudaEventDestroy(b.win_free[1]);
    }
    delete sv;
}

}  // extern "C"
