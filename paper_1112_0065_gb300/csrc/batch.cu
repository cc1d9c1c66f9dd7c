// Multi-beam batches: every output tile of every beam's gulp in one launch of
// a persistent kernel (one CTA per resident slot, tiles taken from a global
// atomic work counter), optionally captured once in a CUDA graph.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "dd_internal.h"
#include "tiled_tile.cuh"  // BatchDesc, TiledArgs, kThreads

namespace dd {

using namespace tiled;

struct Batch {
    TiledShape shape;
    bool big = false;
    BatchKernelFn kernel = nullptr;
    std::vector<Plan *> plans;  // plans whose tables the descriptors point at
    size_t smem = 0;
    int grid = 0;
    BatchDesc host;
    BatchDesc *desc = nullptr;
    unsigned long long *counter = nullptr;
    bool use_graph = false;
    cudaGraphExec_t exec = nullptr;
};

static dd_status fill_desc(Batch *b, int nbeams, const dd_beam *beams) {
    if (nbeams < 1 || nbeams > DD_BATCH_MAX_BEAMS || !beams)
        return fail(DD_ERR_INVALID_ARG, "nbeams must be 1..%d", DD_BATCH_MAX_BEAMS);
    BatchDesc &h = b->host;
    memset(&h, 0, sizeof(h));
    h.nbeams = nbeams;
    long long tiles = 0;
    size_t smem = 0;
    const int D = kWarps * b->shape.dms_per_warp;
    const long long T = 16LL * 32 * b->shape.words_per_lane;
    for (int i = 0; i < nbeams; ++i) {
        Plan *p = reinterpret_cast<Plan *>(beams[i].plan);
        if (!p) return fail(DD_ERR_INVALID_ARG, "beam %d has no plan", i);
        if (p->kernel == DD_KERNEL_SIMPLE) return fail(DD_ERR_INVALID_ARG, "beam %d's plan uses the simple kernel", i);
        if ((p->nchan >= 2048) != b->big)
            return fail(DD_ERR_INVALID_ARG, "beams must all have < 2048 or all >= 2048 channels");
        dd_status st = check_exec_args(p, beams[i].d_in, beams[i].ld_in_bytes, beams[i].nsamp_in, beams[i].d_out,
                                       beams[i].ld_out);
        if (st != DD_OK) return st;
        st = ensure_shape_table(p, b->shape);
        if (st != DD_OK) return st;
        const ShapeTable &tb = p->tables.at(shape_key(b->shape));
        TiledArgs &a = h.beam[i];
        a.in = reinterpret_cast<const uint32_t *>(beams[i].d_in);
        a.ld_w = (long long)(beams[i].ld_in_bytes / 4);
        a.tab = tb.tab;
        a.wsrel = tb.wsrel;
        a.nchan = p->nchan;
        a.ndm = p->ndm;
        a.nout = (long long)beams[i].nsamp_in - p->maxdelay;
        a.out = beams[i].d_out;
        a.ld_out = (long long)beams[i].ld_out;
        a.slot = tb.slot;
        a.n_dmb = tb.n_dmb;
        st = tile_error_word(&a.err);
        if (st != DD_OK) return st;
        a.poll_limit = tiled::kStagePollLimit;
        h.tile_start[i] = tiles;
        tiles += ((a.nout + T - 1) / T) * (long long)a.n_dmb;
        smem = std::max(smem, tiled_smem_bytes(p, tb, D));
    }
    h.tile_start[nbeams] = tiles;
    h.ntiles = tiles;
    if (smem > b->smem) return fail(DD_ERR_INVALID_ARG, "beams need more shared memory than the batch was sized for");
    // the plans' tables must outlive this batch's descriptors (the autotuner
    // keeps every table of a plan with live batches)
    for (Plan *p : b->plans) --p->live_batches;
    b->plans.clear();
    for (int i = 0; i < nbeams; ++i) {
        Plan *p = reinterpret_cast<Plan *>(beams[i].plan);
        if (std::find(b->plans.begin(), b->plans.end(), p) == b->plans.end()) {
            b->plans.push_back(p);
            ++p->live_batches;
        }
    }
    return DD_OK;
}

static void free_batch(Batch *b) {
    if (!b) return;
    for (Plan *p : b->plans) --p->live_batches;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->desc) cudaFree(b->desc);
    if (b->counter) cudaFree(b->counter);
    delete b;
}

}  // namespace dd

using namespace dd;

extern "C" {

dd_status dd_batch_create(dd_batch **out, int nbeams, const dd_beam *beams, int use_graph) {
    if (!out) return fail(DD_ERR_INVALID_ARG, "NULL batch pointer");
    *out = nullptr;
    if (nbeams < 1 || nbeams > DD_BATCH_MAX_BEAMS || !beams || !beams[0].plan)
        return fail(DD_ERR_INVALID_ARG, "nbeams must be 1..%d with a plan per beam", DD_BATCH_MAX_BEAMS);
    Batch *b = new (std::nothrow) Batch();
    if (!b) return fail(DD_ERR_NOMEM, "host allocation failed");
    const Plan *p0 = reinterpret_cast<const Plan *>(beams[0].plan);
    b->shape = p0->shape;
    b->big = p0->nchan >= 2048;
    b->kernel = batch_kernel(b->shape, b->big);
    b->use_graph = use_graph != 0;
    if (!b->kernel) {
        free_batch(b);
        return fail(DD_ERR_INVALID_ARG, "unsupported tile shape");
    }
    // size shared memory for the largest beam, with room to grow to the opt-in limit
    b->smem = 227 * 1024;
    dd_status st = fill_desc(b, nbeams, beams);
    if (st != DD_OK) {
        free_batch(b);
        return st;
    }
    size_t need = 0;
    for (int i = 0; i < nbeams; ++i) {
        const Plan *p = reinterpret_cast<const Plan *>(beams[i].plan);
        const ShapeTable &tb = p->tables.at(shape_key(b->shape));
        need = std::max(need, tiled_smem_bytes(p, tb, kWarps * b->shape.dms_per_warp));
    }
    b->smem = need;
    cudaError_t e = cudaFuncSetAttribute(b->kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
    int dev = 0, sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, b->kernel, kThreads, b->smem);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
    if (e == cudaSuccess) e = cudaMalloc(&b->desc, sizeof(BatchDesc));
    if (e == cudaSuccess) e = cudaMalloc(&b->counter, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpy(b->desc, &b->host, sizeof(BatchDesc), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        st = cuda_fail(e, "batch setup");
        free_batch(b);
        return st;
    }
    b->grid = sms * per_sm;
    if (b->use_graph) {
        cudaStream_t cs = nullptr;
        cudaGraph_t g = nullptr;
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaMemsetAsync(b->counter, 0, sizeof(unsigned long long), cs);
            b->kernel<<<b->grid, kThreads, b->smem, cs>>>(b->desc, b->counter);
            e = cudaStreamEndCapture(cs, &g);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (cs) cudaStreamDestroy(cs);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "capturing the batch graph");
            free_batch(b);
            return st;
        }
    }
    *out = reinterpret_cast<dd_batch *>(b);
    return DD_OK;
}

dd_status dd_batch_set(dd_batch *batch, int nbeams, const dd_beam *beams, void *stream) {
    Batch *b = reinterpret_cast<Batch *>(batch);
    if (!b) return fail(DD_ERR_INVALID_ARG, "NULL batch");
    dd_status st = fill_desc(b, nbeams, beams);
    if (st != DD_OK) return st;
    return cuda_fail(cudaMemcpyAsync(b->desc, &b->host, sizeof(BatchDesc), cudaMemcpyHostToDevice,
                                     (cudaStream_t)stream),
                     "uploading batch descriptors");
}

dd_status dd_batch_launch(dd_batch *batch, void *stream) {
    Batch *b = reinterpret_cast<Batch *>(batch);
    if (!b) return fail(DD_ERR_INVALID_ARG, "NULL batch");
    cudaStream_t s = (cudaStream_t)stream;
    if (b->use_graph) return cuda_fail(cudaGraphLaunch(b->exec, s), "cudaGraphLaunch");
    DD_CUDA_TRY(cudaMemsetAsync(b->counter, 0, sizeof(unsigned long long), s));
    b->kernel<<<b->grid, kThreads, b->smem, s>>>(b->desc, b->counter);
    return cuda_fail(cudaGetLastError(), "dd_batch_kernel launch");
}

dd_status dd_batch_info(const dd_batch *batch, int *nbeams, long long *ntiles, int *grid, int *dms_per_block,
                        int *words_per_thread) {
    const Batch *b = reinterpret_cast<const Batch *>(batch);
    if (!b) return fail(DD_ERR_INVALID_ARG, "NULL batch");
    if (nbeams) *nbeams = b->host.nbeams;
    if (ntiles) *ntiles = b->host.ntiles;
    if (grid) *grid = b->grid;
    if (dms_per_block) *dms_per_block = kWarps * b->shape.dms_per_warp;
    if (words_per_thread) *words_per_thread = b->shape.words_per_lane;
    return DD_OK;
}

void dd_batch_destroy(dd_batch *batch) { free_batch(reinterpret_cast<Batch *>(batch)); }

dd_status dd_execute_batch(int nbeams, const dd_beam *beams, void *stream) {
    dd_batch *b = nullptr;
    dd_status st = dd_batch_create(&b, nbeams, beams, 0);
    if (st != DD_OK) return st;
    st = dd_batch_launch(b, stream);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    dd_batch_destroy(b);
    if (st != DD_OK) return st;
    return cuda_fail(e, "waiting for the batch");
}

}  // extern "C"
