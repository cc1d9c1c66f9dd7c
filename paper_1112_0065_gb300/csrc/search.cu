// Search stage after dedispersion (paper Section 2.3): baseline removal,
// boxcar matched filtering over a list of widths, a sigma cut and grouping of
// contiguous above-threshold cells into events, and DM-time snippets around
// each event for the classifier.
//
// Kernels (all exact integer arithmetic up to the S/N division):
//  * dd_median_kernel   every lane keeps a histogram of the sliding window
//                    [t-half, t+half) of its own row segment in shared memory
//                    and walks the lower median as the window moves; writes
//                    y = x - median and adds sum(y^2) to the row total (int64).
//  * dd_xprefix_kernel, dd_mean_apply_kernel  the paper's running mean instead
//                    (an option): row prefix sums, then x minus the window mean
//                    rounded half up.
//  * dd_mf_kernel       a CTA loads a tile of y plus the widest boxcar's halo,
//                    prefix-sums it in shared memory, and for every sample
//                    decides with integer thresholds whether some width reaches
//                    the S/N cut; hot cells get their best S/N and width and a
//                    bit in the row's hot bitmask.
//  * runs/vunion/compress/ids/group_reduce kernels: 4-connected groups in
//                    (DM, time) from runs of hot cells along time joined across
//                    rows by union-find (roots = smallest run start, so the
//                    result is deterministic); one record per group at its best
//                    cell.
//  * mark/count_marks/scan_chunks/write_marks: the records in (DM, time) order.
//  * dd_snippet_kernel  64 DM rows x 64 bins of w samples around each event, each
//                    bin the S/N of its boxcar, rounded to bfloat16.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "dd_internal.h"

namespace dd {
namespace {

constexpr int kMaxWidths = 16;
constexpr int kMfThreads = 256;
constexpr int kMfTile = 4096;
constexpr int kCompactThreads = 256;
constexpr int kCompactChunk = 1 << 16;  // cells per compaction chunk
constexpr unsigned kUnionCap = 1u << 22;  // bound on union-find retries per edge

struct DevState {
    unsigned long long nhot;
    unsigned int nroots;
    unsigned int err;  // bit 0: value beyond histogram; bit 2: union cap hit
    unsigned long long nrebuild;  // median histograms recounted from their window
};

struct SearchCfgDev {
    int nw;
    int widths[kMaxWidths];
    unsigned wmask;  // bit j: width 2^j is searched (widths are powers of two <= 1024)
};
constexpr int kPows = 11;  // possible widths 2^0 .. 2^10

// ---------------------------------------------------------------------------
// baseline: sliding lower median by histogram walk
// ---------------------------------------------------------------------------

// Each lane walks the lower median of one row segment of h = half_window
// outputs; lane slot g = d * nseg + s owns outputs [s*h, min(n, (s+1)*h)) of
// row d.  The window [t-h, t+h) of any of them lies in segments s-1..s+1, so
// the three value streams a lane needs at step t (x[t-h] leaving, x[t], and
// x[t+h] entering the window) are, at the same offset, the values of slots
// g-1, g and g+1.  A warp therefore stages, 32 steps at a time, the values of
// the 34 slots g0-1 .. g0+32 with one coalesced load per slot, and each lane
// reads its three streams from that tile.
//
// A lane's histogram has kMedBins 32-bit counts (words interleaved across
// lanes so each lane stays in its own bank): bin 0 counts
// values below `base`, bins 1..kMedBins-2 the values base..base+kMedBins-3,
// and the last bin values above; the median walks over the inner bins and the
// lane rebuilds its histogram around the median when it reaches an edge.
// `below` counts the window's values < m and `hm` those equal to m.
constexpr int kMedBins = 64;
constexpr int kMedWords = kMedBins;  // one count per word
constexpr int kMedInner = kMedBins - 2;  // values covered by the inner bins
constexpr int kMedStage = 34;            // staged slots per warp
constexpr int kTileStride = 33;          // padded tile row (conflict-free)
constexpr uint16_t kNoValue = 0xFFFFu;   // values are clipped to 3*nchan <= 65532 first

struct MedSlot {
    long long xoff;  // element offset of the slot's first value in x
    int yoff;        // element offset of its first output in y
    int len;         // values in the slot (0: no slot)
};

__device__ __forceinline__ int med_bin(int v, int base) { return min(max(v - base + 1, 0), kMedBins - 1); }
// Bin of the sweep: like med_bin for the inner bins and bin 0; values below
// base - 1 land in the last bin instead of the first.
__device__ __forceinline__ int sweep_bin(int v, int base) {
    return (int)min((unsigned)(v - base + 1), (unsigned)(kMedBins - 1));
}
__device__ __forceinline__ int hget(const uint32_t *H, int b, int lane) { return (int)H[b * 32 + lane]; }
// A shared-memory atomic add whose result is unused: the update leaves the
// lane's dependency chain (the walk's later reads of its own column see it).
__device__ __forceinline__ void hadd(uint32_t *H, int b, int lane, uint32_t one) {
    atomicAdd(&H[b * 32 + lane], one);  // one = 1 or 0xFFFFFFFF (-1)
}

// Median of rank r from a complete histogram: -> bin index, count below it, its count.
__device__ __forceinline__ int med_scan(const uint32_t *H, int lane, int r, int &below, int &hm) {
    int cum = 0;
    for (int b = 0; b < kMedBins; ++b) {
        const int c = hget(H, b, lane);
        if (cum + c > r) {
            below = cum;
            hm = c;
            return b;
        }
        cum += c;
    }
    below = cum;
    hm = 0;
    return kMedBins - 1;  // not reached for a consistent histogram
}

// Warp-cooperative rebuild of the histograms of the lanes in `need` (a
// ballot): for each such lane L all 32 lanes read L's window row[lo, hi)
// (clipped to top) with coalesced loads and add it into L's histogram column
// with shared atomics around L's new base; L then takes the median of rank r
// and, when it lands on an edge bin, moves the base and the warp counts again
// (a bounded number of times; `bad` is set if that runs out).  Called by all
// 32 lanes together.
__device__ __forceinline__ void med_coop_rebuild(unsigned need, const uint32_t *__restrict__ x, long long ld_x, int d, long long lo,
                                 long long hi, int top, int r, uint32_t *H, int lane, int &base, int &m, int &below,
                                 int &hm, bool &bad) {
    const int maxbase = max(0, top - (kMedInner - 1));
    while (need) {
        const int L = __ffs(need) - 1;
        need &= need - 1;
        const int dL = __shfl_sync(0xffffffffu, d, L);
        const long long loL = __shfl_sync(0xffffffffu, lo, L), hiL = __shfl_sync(0xffffffffu, hi, L);
        const int rL = __shfl_sync(0xffffffffu, r, L);
        int baseL = __shfl_sync(0xffffffffu, base, L);
        const uint32_t *rowL = x + (long long)dL * ld_x;
        for (int guard = 0; guard < 4096; ++guard) {
            H[lane * 32 + L] = 0u;  // lane L's column: words lane and lane + 32
            H[(lane + 32) * 32 + L] = 0u;
            __syncwarp();
            // eight coalesced loads in flight per round, then their counts
            for (long long i0 = loL; i0 < hiL; i0 += 8 * 32) {
                uint32_t v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const long long i = i0 + 32 * u + lane;
                    v[u] = i < hiL ? __ldg(rowL + i) : 0u;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (i0 + 32 * u + lane < hiL) atomicAdd(&H[med_bin((int)min(v[u], (uint32_t)top), baseL) * 32 + L], 1u);
            }
            __syncwarp();
            int retry = 0;
            if (lane == L) {
                const int b = med_scan(H, lane, rL, below, hm);
                if (b == 0 && baseL > 0) {
                    baseL = max(0, baseL - kMedInner / 2);
                    retry = 1;
                } else if (b == kMedBins - 1 && baseL < maxbase) {
                    baseL = min(maxbase, baseL + kMedInner / 2);
                    retry = 1;
                } else {
                    base = baseL;
                    m = baseL + b - 1;
                    bad |= !(b > 0 && b < kMedBins - 1);
                }
            }
            retry = __shfl_sync(0xffffffffu, retry, L);
            baseL = __shfl_sync(0xffffffffu, baseL, L);
            if (!retry) break;
            if (guard == 4095 && lane == L) bad = true;
            __syncwarp();
        }
    }
}

// Loads of the values of slots g0-1 .. g0+32 at offsets [bt, bt+32): one
// chunk is in flight in registers while the warp works on the previous one.
struct MedPrefetch {
    uint32_t v[kMedStage];
    unsigned long long valid;  // bit j: slot j has a value at this offset
    bool full;                 // every slot has all 32 values (valid unused)
};

// full: bt + 32 <= the shortest of the 34 slots (warp-uniform), so no value
// needs a bounds test.
__device__ __forceinline__ void med_issue(const uint32_t *__restrict__ x, const MedSlot *slot, int bt, int lane,
                                          bool full, MedPrefetch &pf) {
    pf.full = full;
    if (full) {
#pragma unroll
        for (int j = 0; j < kMedStage; ++j) pf.v[j] = __ldg(x + slot[j].xoff + bt + lane);
        return;
    }
    pf.valid = 0;
#pragma unroll
    for (int j = 0; j < kMedStage; ++j) {
        const MedSlot sl = slot[j];
        const bool ok = bt + lane < sl.len;
        pf.v[j] = ok ? __ldg(x + sl.xoff + bt + lane) : 0u;
        pf.valid |= (unsigned long long)ok << j;
    }
}

// Clip the prefetched values to top and store them as tile[j][lane] (NoValue
// where a slot has no value).  Returns true when a value above top was seen.
__device__ __forceinline__ bool med_commit(const MedPrefetch &pf, uint32_t top, uint16_t *tile, int lane) {
    bool over = false;
    if (pf.full) {
#pragma unroll
        for (int j = 0; j < kMedStage; ++j) {
            over |= pf.v[j] > top;
            tile[j * kTileStride + lane] = (uint16_t)min(pf.v[j], top);
        }
        return over;
    }
#pragma unroll
    for (int j = 0; j < kMedStage; ++j) {
        const bool ok = (pf.valid >> j) & 1ull;
        over |= ok && pf.v[j] > top;
        tile[j * kTileStride + lane] = ok ? (uint16_t)min(pf.v[j], top) : kNoValue;
    }
    return over;
}

// Shared memory of one warp: the histograms, the value tile, then (WIDE) the
// int32 output tile or (narrow: |y| <= top <= 32767) slot g0-1's counts --
// narrow outputs go back into the value tile as int16.
template <bool WIDE>
constexpr size_t med_smem_bytes() {
    return (size_t)kMedWords * 32 * 4 + ((size_t)kMedStage * kTileStride * 2 + 3) / 4 * 4 +
           (WIDE ? (size_t)32 * kTileStride * 4 : (size_t)kMedWords * 4);
}

template <bool WIDE>
__global__ void __launch_bounds__(32, WIDE ? 14 : 16) dd_median_kernel(const uint32_t *__restrict__ x, long long ld_x,
                                                                      int ndm, long long n, int h, int nbins,
                                                                      int32_t *__restrict__ y, long long ld_y,
                                                                      unsigned long long *__restrict__ sumsq,
                                                                      DevState *st) {
    extern __shared__ __align__(16) uint32_t H[];  // kMedWords x 32 lanes, then the tiles
    uint16_t *tile = reinterpret_cast<uint16_t *>(H + kMedWords * 32);                   // [34][33] values
    // after the value tile: [32][33] int32 outputs (WIDE) or slot g0-1's counts
    uint32_t *after = H + kMedWords * 32 + (kMedStage * kTileStride * 2 + 3) / 4;
    int32_t *t_y = reinterpret_cast<int32_t *>(after);
    __shared__ MedSlot slot[kMedStage];
    const int lane = threadIdx.x;
    const long long nseg = (n + h - 1) / h;
    const long long nslots = (long long)ndm * nseg;
    const long long g0 = (long long)blockIdx.x * 32;
    for (int j = lane; j < kMedStage; j += 32) {
        const long long gj = g0 - 1 + j;
        MedSlot sl{0, 0, 0};
        if (gj >= 0 && gj < nslots) {
            const long long dj = gj / nseg, sj = gj % nseg;
            sl.xoff = dj * ld_x + sj * h;
            sl.yoff = (int)(dj * ld_y + sj * h);
            sl.len = (int)min((long long)h, n - sj * h);
        }
        slot[j] = sl;
    }
    __syncwarp();
    // shortest staged slot (0 where a slot is missing) and shortest output slot
    const int minlen_all = __reduce_min_sync(0xffffffffu, (unsigned)min(slot[lane].len, lane < 2 ? slot[lane + 32].len
                                                                                                 : slot[lane].len));
    const int minlen_out = __reduce_min_sync(0xffffffffu, (unsigned)slot[lane + 1].len);
    const long long g = g0 + lane;
    const bool active = g < nslots;
    const int d = active ? (int)(g / nseg) : 0;
    const long long s = active ? g % nseg : 0;
    const long long s0 = s * h;
    const int len = slot[lane + 1].len;       // outputs of this lane (0 when inactive)
    const bool has_prev = s > 0;              // x[t-h] exists for every t of the segment
    const bool has_next = s + 1 < nseg;       // x[t+h] lies in the next slot of the same row
    const uint32_t *row = x + (long long)d * ld_x;
    const int top = nbins - 1;
    const int maxbase = max(0, top - (kMedInner - 1));
    const int seglen_max = __reduce_max_sync(0xffffffffu, len);  // steps of the sweep
    // steps of the build: the previous slot (h values) and this one
    const int build_steps = max(seglen_max, __reduce_max_sync(0xffffffffu, has_prev ? h : 0));
    const int nb = (build_steps + 31) / 32, ns = (seglen_max + 31) / 32;
    bool bad = false;

    // first window [s0-h, s0+h) = slot g-1 + slot g.  Every lane counts its
    // own slot and then adds lane l-1's counts (lane 0 those of slot g0-1,
    // counted by the whole warp into Hx), so the warp shares one histogram
    // range: around the median of the lanes' estimates, each the median of
    // 7 values spread over the lane's window.
    const long long lo = max(0LL, s0 - h), hi = min(n, s0 + h);
    int wsize = (int)(hi - lo);
    int est = -1;
    if (active) {
        int a[7];
#pragma unroll
        for (int j = 0; j < 7; ++j) a[j] = (int)min(__ldg(row + lo + (hi - 1 - lo) * j / 6), (uint32_t)top);
#pragma unroll
        for (int p = 0; p < 7; ++p)
#pragma unroll
            for (int j = p & 1; j + 1 < 7; j += 2) {
                const int lo2 = min(a[j], a[j + 1]), hi2 = max(a[j], a[j + 1]);
                a[j] = lo2;
                a[j + 1] = hi2;
            }
        est = a[3];
    }
    int base = 0;
    {
        int lt = 0, le = 0;
        for (int k = 0; k < 32; ++k) {
            const int o = __shfl_sync(0xffffffffu, est, k);
            lt += (o >= 0) & (o < est);
            le += (o >= 0) & (o <= est);
        }
        const int want = (__popc(__ballot_sync(0xffffffffu, est >= 0)) - 1) >> 1;
        const unsigned pick = __ballot_sync(0xffffffffu, est >= 0 && lt <= want && want < le);
        const int mest = pick ? __shfl_sync(0xffffffffu, est, __ffs(pick) - 1) : 0;
        base = max(0, min(maxbase, mest - kMedInner / 2));
    }
    const bool prev0 = __shfl_sync(0xffffffffu, has_prev, 0);  // slot g0-1 is in lane 0's row
    uint32_t *Hx = after;  // slot g0-1's counts (WIDE: in t_y, free until the sweep)
    Hx[lane] = 0u;
    Hx[lane + 32] = 0u;
    for (int w = 0; w < kMedWords; ++w) H[w * 32 + lane] = 0u;
    int r = (wsize - 1) >> 1;
    int m = 0, below = 0, hm = 0;
    unsigned long long ssq = 0;

    MedPrefetch pf;
    med_issue(x, slot, 0, lane, 32 <= minlen_all, pf);
    for (int c = 0; c < nb + ns; ++c) {
        const bool building = c < nb;
        const int bt = (building ? c : c - nb) * 32;
        bad |= med_commit(pf, (uint32_t)top, tile, lane);
        __syncwarp();
        if (c + 1 < nb + ns) {
            const int bn = (c + 1 < nb ? c + 1 : c + 1 - nb) * 32;
            med_issue(x, slot, bn, lane, bn + 32 <= minlen_all, pf);
        }
        if (building) {
            // ---- histograms of the lanes' slots and of slot g0-1
            if (active) {
#pragma unroll 4
                for (int i = 0; i < 32; ++i) {
                    const int vc = tile[(lane + 1) * kTileStride + i];
                    hadd(H, med_bin(vc, base), lane, (uint32_t)(vc != kNoValue));
                }
            }
            if (prev0) {
                const int v0 = tile[lane];
                if (v0 != kNoValue) {
                    const int b = med_bin(v0, base);
                    atomicAdd(&Hx[b], 1u);
                }
            }
            if (c == nb - 1) {
                // window = own slot + previous slot
                __syncwarp();
#pragma unroll 1
                for (int w0 = 0; w0 < kMedWords; w0 += 16) {
                    uint32_t nbh[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k) nbh[k] = lane == 0 ? Hx[w0 + k] : H[(w0 + k) * 32 + lane - 1];
                    __syncwarp();
                    if (has_prev) {
#pragma unroll
                        for (int k = 0; k < 16; ++k) H[(w0 + k) * 32 + lane] += nbh[k];
                    }
                    __syncwarp();
                }
                bool need = false;
                if (active) {
                    const int b = med_scan(H, lane, r, below, hm);
                    m = base + b - 1;
                    if (b == 0 || b == kMedBins - 1) {
                        base = max(0, min(maxbase, (b == 0 ? base - kMedInner : base + kMedInner)));
                        need = true;
                    }
                }
                __syncwarp();
                const unsigned nmask = __ballot_sync(0xffffffffu, need);
                if (nmask) {
                    if (lane == 0) atomicAdd(&st->nrebuild, (unsigned long long)__popc(nmask));
                    med_coop_rebuild(nmask, x, ld_x, d, lo, hi, top, r, H, lane, base, m, below, hm, bad);
                }
            }
            __syncwarp();
            continue;
        }
        // ---- sweep: output y[t] = x[t] - m, then move the window to t+1 (also
        // after a segment's last output: harmless, the state is dropped)
        {
            const int nst = active ? min(32, len - bt) : 0;
            const int nst_w = __reduce_max_sync(0xffffffffu, nst);  // the warp steps together
            int32_t yprev = 0;
#pragma unroll 2
            for (int i = 0; i < nst_w; ++i) {
                bool need = false;
                if (i < nst) {
                const int vc = tile[(lane + 1) * kTileStride + i];
                const int32_t yv = vc - m;
                if (WIDE) {
                    t_y[lane * kTileStride + i] = yv;
                } else {
                    // column i-1 of the tile was read by every lane before the
                    // previous step's ballot: it takes that step's output
                    if (i > 0) tile[(lane + 1) * kTileStride + i - 1] = (uint16_t)yprev;
                    yprev = yv;
                }
                ssq += (uint32_t)yv * (uint32_t)yv;  // |y| <= 65532: the square fits 32 bits
                const int vo = has_prev ? tile[lane * kTileStride + i] : kNoValue;
                const int vi = has_next ? tile[(lane + 2) * kTileStride + i] : kNoValue;
                // Branch-free.  The sweep reads only the inner bins, so values
                // outside them (and kNoValue, which lies above every median)
                // all go to the last bin, whose count it never reads.
                hadd(H, sweep_bin(vo, base), lane, 0xFFFFFFFFu);
                hadd(H, sweep_bin(vi, base), lane, 1u);
                wsize += (vi != kNoValue) - (vo != kNoValue);
                below += (vi < m) - (vo < m);
                hm += (vi == m) - (vo == m);
                r = (wsize - 1) >> 1;
                if (below > r || below + hm <= r) {  // the median moves (rarely)
                    bool rebuild = false;
                    while (below > r) {
                        if (m <= base) {
                            rebuild = true;
                            break;
                        }
                        --m;
                        hm = hget(H, m - base + 1, lane);
                        below -= hm;
                    }
                    while (!rebuild && below + hm <= r) {
                        if (m >= base + kMedInner - 1) {
                            rebuild = true;
                            break;
                        }
                        below += hm;
                        ++m;
                        hm = hget(H, m - base + 1, lane);
                    }
                    if (rebuild) {
                        base = max(0, min(maxbase, m - kMedInner / 2));
                        need = true;
                    }
                }
                }
                const unsigned nmask = __ballot_sync(0xffffffffu, need);
                if (nmask) {
                    if (lane == 0) atomicAdd(&st->nrebuild, (unsigned long long)__popc(nmask));
                    const long long t1 = s0 + bt + i + 1;
                    med_coop_rebuild(nmask, x, ld_x, d, max(0LL, t1 - h), min(n, t1 + h), top, r, H, lane, base, m,
                                     below, hm, bad);
                }
            }
            if (!WIDE && nst > 0) tile[(lane + 1) * kTileStride + nst - 1] = (uint16_t)yprev;
        }
        __syncwarp();
        // coalesced write-back of the 32 outputs of every lane
        auto yval = [&](int j) -> int32_t {
            return WIDE ? t_y[j * kTileStride + lane] : (int32_t)(int16_t)tile[(j + 1) * kTileStride + lane];
        };
        if (bt + 32 <= minlen_out) {
#pragma unroll 8
            for (int j = 0; j < 32; ++j) y[slot[j + 1].yoff + bt + lane] = yval(j);
        } else {
#pragma unroll 4
            for (int j = 0; j < 32; ++j) {
                const MedSlot sl = slot[j + 1];
                if (bt + lane < sl.len) y[sl.yoff + bt + lane] = yval(j);
            }
        }
        __syncwarp();
    }
    if (active) atomicAdd(sumsq + d, ssq);
    if (bad) atomicOr(&st->err, 1u);
}

// ---------------------------------------------------------------------------
// baseline, paper form: running mean (rounded half up) from row prefix sums
// ---------------------------------------------------------------------------

// Tile-local exclusive prefix of x (values clipped to top) and the tile's
// total: a CTA stages kMfTile samples, each thread sums 16 consecutive ones,
// a block scan of the thread totals gives its offset.
__global__ void __launch_bounds__(256) dd_xprefix_kernel(const uint32_t *__restrict__ x, long long ld_x, long long n,
                                                         uint32_t top, int32_t *__restrict__ pre,
                                                         long long *__restrict__ tile_sum, int ntiles,
                                                         DevState *st) {
    // element i at i + i/16: a thread's 16 consecutive elements start at 17*tid,
    // so the scan's reads and writes hit 32 distinct banks
    __shared__ uint32_t xs[kMfTile + kMfTile / 16];
    __shared__ int32_t s_warp[8];
    const int d = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long t0 = (long long)blockIdx.x * kMfTile;
    const uint32_t *row = x + (long long)d * ld_x;
    bool over = false;
    for (int i = tid; i < kMfTile; i += 256) {
        uint32_t v = 0;
        if (t0 + i < n) {
            v = __ldg(row + t0 + i);
            over |= v > top;
            v = min(v, top);
        }
        xs[i + (i >> 4)] = v;
    }
    if (__any_sync(0xffffffffu, over) && lane == 0) atomicOr(&st->err, 1u);
    __syncthreads();
    int32_t loc[16];
    int32_t tot = 0;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        loc[q] = tot;
        tot += (int32_t)xs[17 * tid + q];
    }
    int32_t incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    int32_t off = incl - tot;
    for (int w = 0; w < warp; ++w) off += s_warp[w];
    if (tid == 255) tile_sum[(long long)d * ntiles + blockIdx.x] = off + tot;
    __syncthreads();
    // back through shared memory for coalesced stores
#pragma unroll
    for (int q = 0; q < 16; ++q) xs[17 * tid + q] = (uint32_t)(loc[q] + off);
    __syncthreads();
    int32_t *prow = pre + (long long)d * n;
    for (int i = tid; i < kMfTile; i += 256)
        if (t0 + i < n) prow[t0 + i] = (int32_t)xs[i + (i >> 4)];
}

// floor(a / m) for a < 2^32 and 1 <= m < 2^16 from rm = 1/m rounded to
// nearest: the float estimate a*rm is within 2^-6 of a/m (three roundings
// of at most 2^-23 relative each, a/m < 2^16), so its truncation is off by
// at most one, which one exact integer remainder corrects.
__device__ __forceinline__ uint32_t udiv_small(uint32_t a, uint32_t m, float rm) {
    uint32_t q = __float2uint_rz(__uint2float_rz(a) * rm);
    const long long r = (long long)a - (long long)q * m;
    if (r < 0) --q;
    else if (r >= (long long)m) ++q;
    return q;
}

// y[t] = x[t] - floor((S + floor(m/2)) / m) for the window sum S of its m
// values (= the mean rounded half up; S < 2^32 since m <= 65534 and x <=
// 65532), and the row's sum of y^2.  A block takes kMeanCells consecutive
// outputs of a row, a thread every 256th.  Prefix values are used modulo 2^32:
// a window sum is below 2^32, so the difference of the low words is exact.
constexpr int kMeanCells = 2048;
__global__ void __launch_bounds__(256) dd_mean_apply_kernel(const uint32_t *__restrict__ x, long long ld_x, long long n,
                                                            long long h, uint32_t top,
                                                            const int32_t *__restrict__ pre,
                                                            const long long *__restrict__ tile_off,
                                                            const long long *__restrict__ tile_sum, int ntiles,
                                                            int32_t *__restrict__ y, long long ld_y,
                                                            unsigned long long *__restrict__ sumsq) {
    const int d = blockIdx.y;
    const int32_t *prow = pre + (long long)d * n;
    const long long *orow = tile_off + (long long)d * ntiles;
    const uint32_t *xrow = x + (long long)d * ld_x;
    int32_t *yrow = y + (long long)d * ld_y;
    const int ni = (int)n, hi32 = (int)h;  // n < 2^31 (cells are int32 indices)
    const uint32_t p_end = (uint32_t)(orow[ntiles - 1] + tile_sum[(long long)d * ntiles + ntiles - 1]);
    const uint32_t m_full = (uint32_t)min(2LL * h, n);
    const float rm_full = __frcp_rn((float)m_full);
    unsigned long long sq = 0;
    const int t0 = blockIdx.x * kMeanCells + threadIdx.x;
#pragma unroll 4
    for (int j = 0; j < kMeanCells / 256; ++j) {
        const int t = t0 + 256 * j;
        if (t >= ni) break;
        const int lo = max(0, t - hi32), hi = min(ni, t + hi32);
        const uint32_t p_hi = hi == ni ? p_end : (uint32_t)orow[hi / kMfTile] + (uint32_t)prow[hi];
        const uint32_t p_lo = (uint32_t)orow[lo / kMfTile] + (uint32_t)prow[lo];
        const uint32_t S = p_hi - p_lo;
        const uint32_t m = (uint32_t)(hi - lo);
        const float rm = m == m_full ? rm_full : __frcp_rn((float)m);
        const uint32_t mean = udiv_small(S + m / 2, m, rm);
        const int32_t yv = (int32_t)min(__ldg(xrow + t), top) - (int32_t)mean;
        yrow[t] = yv;
        sq += (unsigned long long)((long long)yv * yv);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if ((threadIdx.x & 31) == 0 && sq) atomicAdd(sumsq + d, sq);
}

// Fused form of the same baseline, used when a tile's window span fits in
// shared memory: a CTA takes kMeanTile consecutive outputs of a row, stages
// the row's values over [t0 - h, t0 + kMeanTile + h) (clipped to the row and
// to top), forms their exclusive prefix P in shared memory (32 values per
// thread per pass, one padding word per 32 so the passes are free of bank
// conflicts), and writes y[t] = x[t] - floor((S + floor(m/2)) / m) with
// S = P[hi] - P[lo] for the window [lo, hi) of t and x[t] = P[t+1] - P[t], and
// the row's sum of y^2.  No row-wide prefix goes through memory.
constexpr int kMeanTile = 8192;
constexpr int kMeanThreads = 512;
constexpr int kMeanPass = 32 * kMeanThreads;  // span values per scan pass
__host__ __device__ constexpr int mean_pad(int i) { return i + (i >> 5); }
inline size_t mean_fused_smem(long long h) {
    const long long span = kMeanTile + 2 * h;
    return (size_t)(mean_pad((int)span) + 1) * 4;
}
constexpr size_t kMeanFusedSmemMax = 200 * 1024;

__global__ void __launch_bounds__(kMeanThreads) dd_mean_fused_kernel(const uint32_t *__restrict__ x, long long ld_x,
                                                                     long long n, long long h, uint32_t top,
                                                                     int32_t *__restrict__ y, long long ld_y,
                                                                     unsigned long long *__restrict__ sumsq,
                                                                     DevState *st) {
    extern __shared__ __align__(16) uint32_t Pm[];
    __shared__ uint32_t s_warp[kMeanThreads / 32];
    __shared__ uint32_t s_carry;
    const int d = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long t0 = (long long)blockIdx.x * kMeanTile;
    const long long lo0 = max(0LL, t0 - h), hi0 = min(n, t0 + kMeanTile + h);
    const int L = (int)(hi0 - lo0);
    const uint32_t *row = x + (long long)d * ld_x + lo0;
    bool over = false;
    // 16-byte loads when the span starts on a 16-byte boundary (4 values at
    // i..i+3 never straddle a padding word), then the ragged rest one by one
    const int L4 = (reinterpret_cast<uintptr_t>(row) & 15u) == 0 ? L / 4 : 0;
    for (int q = tid; q < L4; q += kMeanThreads) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(row) + q);
        over |= v.x > top || v.y > top || v.z > top || v.w > top;
        uint32_t *dst = Pm + mean_pad(4 * q);
        dst[0] = min(v.x, top);
        dst[1] = min(v.y, top);
        dst[2] = min(v.z, top);
        dst[3] = min(v.w, top);
    }
    for (int i = 4 * L4 + tid; i < L; i += kMeanThreads) {
        const uint32_t v = __ldg(row + i);
        over |= v > top;
        Pm[mean_pad(i)] = min(v, top);
    }
    if (__any_sync(0xffffffffu, over) && lane == 0) atomicOr(&st->err, 1u);
    if (tid == 0) s_carry = 0u;
    __syncthreads();
    for (int c0 = 0; c0 < L; c0 += kMeanPass) {
        const int b = c0 + 32 * tid;
        uint32_t v[32];
        uint32_t tot = 0;
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            v[q] = b + q < L ? Pm[mean_pad(b + q)] : 0u;
            const uint32_t e = tot;
            tot += v[q];
            v[q] = e;
        }
        uint32_t incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        uint32_t off = s_carry + incl - tot;
        for (int w = 0; w < warp; ++w) off += s_warp[w];
#pragma unroll
        for (int q = 0; q < 32; ++q)
            if (b + q < L) Pm[mean_pad(b + q)] = v[q] + off;
        __syncthreads();
        if (tid == kMeanThreads - 1) s_carry = off + tot;
        __syncthreads();
    }
    if (tid == 0) Pm[mean_pad(L)] = s_carry;
    __syncthreads();
    const long long m_full = min(2LL * h, n);
    const float rm_full = __frcp_rn((float)m_full);
    const int nt = (int)min((long long)kMeanTile, n - t0);
    int32_t *yrow = y + (long long)d * ld_y + t0;
    unsigned long long sq = 0;
    for (int j = tid; j < nt; j += kMeanThreads) {
        const long long t = t0 + j;
        const int lo = (int)(max(0LL, t - h) - lo0), hi = (int)(min(n, t + h) - lo0), c = (int)(t - lo0);
        const uint32_t S = Pm[mean_pad(hi)] - Pm[mean_pad(lo)];
        const uint32_t m = (uint32_t)(hi - lo);
        const float rm = m == (uint32_t)m_full ? rm_full : __frcp_rn((float)m);
        const uint32_t mean = udiv_small(S + m / 2, m, rm);
        const int32_t xv = (int32_t)(Pm[mean_pad(c + 1)] - Pm[mean_pad(c)]);
        const int32_t yv = xv - (int32_t)mean;
        yrow[j] = yv;
        sq += (unsigned long long)((long long)yv * yv);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (lane == 0 && sq) atomicAdd(sumsq + d, sq);
}

// ---------------------------------------------------------------------------
// matched filter + sigma cut
// ---------------------------------------------------------------------------

// Per (row, width): the denominator float(sigma*sqrt(w)) and the smallest
// boxcar sum S whose S/N, float(S)/den rounded to nearest, reaches thresh.
// The rounded quotient never decreases as S grows, so a cell is hot exactly
// when some S_w >= T_w, decided with integer compares.
__global__ void dd_thresh_kernel(const unsigned long long *__restrict__ sumsq, long long n, const SearchCfgDev cfg,
                                 float thresh, int ndm, float *__restrict__ den, int32_t *__restrict__ tmin) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ndm * cfg.nw) return;
    const int d = i / cfg.nw, k = i % cfg.nw;
    const unsigned long long ss = sumsq[d];
    const double sigma = sqrt((double)ss / (double)n);
    const float dn = (float)(sigma * sqrt((double)cfg.widths[k]));
    den[i] = dn;
    int32_t T = 0x7fffffff;  // a constant row never reaches the threshold
    if (ss != 0ULL) {
        long long t = (long long)ceil((double)thresh * (double)dn);
        const long long cap = 1LL << 30;
        t = max(-cap, min(cap, t));
        while (t > -cap && (float)(t - 1) / dn >= thresh) --t;
        while (t < cap && !((float)t / dn >= thresh)) ++t;
        T = (int32_t)t;
    }
    tmin[i] = T;
}

// A CTA takes kMfTile samples of one row plus the widest boxcar's halo
// (kMfSpan samples in all), forms the exclusive prefix P in shared memory
// (each thread sums kMfSeg consecutive samples, then a block scan of the
// threads' totals), and tests its cells four at a time: a lane owns four
// consecutive cells, reads P at the cells and at the cells + w with 16-byte
// loads, and compares each boxcar sum S_w = P[t+w] - P[t] with the smallest
// sum reaching the threshold.  Hot cells get their best S/N and width; the
// four-cell nibbles of eight lanes form one word of the row's hot bitmask.
constexpr int kMfSpan = kMfTile + 1024;       // samples loaded per tile (tile + widest boxcar)
constexpr int kMfSeg = kMfSpan / kMfThreads;  // samples per thread in the scan
static_assert(kMfSeg % 4 == 0 && kMfSeg * kMfThreads == kMfSpan, "scan segments of whole int4s");

// a / b rounded to nearest from y = 1/b rounded to nearest (Markstein's
// correction step): q = a*y, r = a - b*q (exact with one fused multiply-add),
// q + r*y.  Correctly rounded for normal a, b and quotients away from the
// overflow and underflow ranges -- here |a| < 2^31 is an integer and b =
// sigma * sqrt(w) lies far from both.
__device__ __forceinline__ float div_rn(float a, float b, float y) {
    const float q = a * y;
    const float r = fmaf(-q, b, a);
    return fmaf(r, y, q);
}

// Hot flags of the four cells t..t+3: some searched width 2^j has
// P[t+i+2^j] - P[t+i] >= tm[j] (and, outside INSIDE tiles, t+i+2^j <= nrem).
// The widths are compile-time offsets; 1 and 2 come from the registers
// p0 = P[t..t+3], p45 = P[t+4..t+5], the others from 16-byte loads.
// ALLW: all 11 widths are searched (wmask = 0x7FF), so no width test is needed.
template <bool INSIDE, bool ALLW>
__device__ __forceinline__ void mf_test4(const int32_t *P, int t, int nrem, unsigned wmask, const int32_t (&tm)[kPows],
                                         int4 p0, int2 p45, bool &h0, bool &h1, bool &h2, bool &h3) {
    if constexpr (INSIDE) {
        // S - T >= 0 for some width <=> the AND of all S - T has its sign bit
        // clear: one add and half a 3-input AND per (cell, width) instead of a
        // compare.  |S| < 2^27 and |T| <= 2^30 (or T = INT_MAX with S = 0 on a
        // constant row), so S - T does not wrap.
        int32_t a0 = -1, a1 = -1, a2 = -1, a3 = -1;
#pragma unroll
        for (int j = 0; j < kPows; ++j) {
            if (!ALLW && !((wmask >> j) & 1u)) continue;
            int4 pw;
            if (j == 0) pw = make_int4(p0.y, p0.z, p0.w, p45.x);
            else if (j == 1) pw = make_int4(p0.z, p0.w, p45.x, p45.y);
            else pw = *reinterpret_cast<const int4 *>(P + t + (1 << j));
            const int32_t T = tm[j];
            a0 &= pw.x - p0.x - T;
            a1 &= pw.y - p0.y - T;
            a2 &= pw.z - p0.z - T;
            a3 &= pw.w - p0.w - T;
        }
        h0 = a0 >= 0;
        h1 = a1 >= 0;
        h2 = a2 >= 0;
        h3 = a3 >= 0;
    } else {
#pragma unroll
    for (int j = 0; j < kPows; ++j) {
        if (!ALLW && !((wmask >> j) & 1u)) continue;
        const int w = 1 << j;
        int4 pw;
        if (j == 0) pw = make_int4(p0.y, p0.z, p0.w, p45.x);
        else if (j == 1) pw = make_int4(p0.z, p0.w, p45.x, p45.y);
        else pw = *reinterpret_cast<const int4 *>(P + t + w);
        const int32_t T = tm[j];
        h0 |= t + w <= nrem && pw.x - p0.x >= T;
        h1 |= t + 1 + w <= nrem && pw.y - p0.y >= T;
        h2 |= t + 2 + w <= nrem && pw.z - p0.z >= T;
        h3 |= t + 3 + w <= nrem && pw.w - p0.w >= T;
    }
    }
}

template <bool ALLW>
__global__ void __launch_bounds__(kMfThreads) dd_mf_kernel(const int32_t *__restrict__ y, long long ld_y, long long n,
                                                        const unsigned long long *__restrict__ sumsq,
                                                        const SearchCfgDev cfg, float thresh,
                                                        float *__restrict__ best, uint16_t *__restrict__ bestw,
                                                        uint32_t *__restrict__ hotbits, int nwr, DevState *st,
                                                        int32_t *__restrict__ pre, long long *__restrict__ tile_sum,
                                                        int ntiles, const float *__restrict__ den_all,
                                                        const int32_t *__restrict__ tmin_all, int full_map) {
    __shared__ __align__(16) int32_t P[kMfSpan];  // exclusive prefix of the tile's samples
    // per-width values indexed by log2(width)
    __shared__ float s_den[kPows];
    __shared__ float s_rcp[kPows];  // 1/den rounded to nearest
    __shared__ int32_t s_tmin[kPows];
    __shared__ int32_t s_warp[kMfThreads / 32];
    __shared__ unsigned s_nhot;
    __shared__ unsigned s_nlist;
    __shared__ uint16_t s_list[kMfTile];  // tile cells whose S/N is computed
    const int d = blockIdx.y;
    const long long t0 = (long long)blockIdx.x * kMfTile;
    const int nw = cfg.nw;
    const unsigned wmask = cfg.wmask;
    const int32_t *row = y + (long long)d * ld_y;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned long long ss = sumsq[d];
    if (tid < kPows) {
        const bool has = (wmask >> tid) & 1u;
        const int k = __popc(wmask & ((1u << tid) - 1u));  // index of width 2^tid in the list
        const float dn = has ? den_all[d * nw + k] : 1.0f;
        s_den[tid] = dn;
        s_rcp[tid] = __frcp_rn(dn);
        s_tmin[tid] = has ? tmin_all[d * nw + k] : 0x7fffffff;
    }
    if (tid == 0) {
        s_nhot = 0;
        s_nlist = 0;
    }
    // samples of the row from t0 (0 past its end): every copy in flight at
    // once.  16-byte cp.async when the whole span lies in the row and starts
    // on a 16-byte boundary; else 4-byte ones (a copy past the end reads
    // nothing and writes 0)
    if (t0 + kMfSpan <= n && ((reinterpret_cast<uintptr_t>(row + t0) & 15u) == 0)) {
#pragma unroll
        for (int q = 0; q < kMfSeg / 4; ++q) {
            const int i = 4 * (tid + q * kMfThreads);
            const unsigned dst = (unsigned)__cvta_generic_to_shared(P + i);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(row + t0 + i) : "memory");
        }
    } else {
#pragma unroll
        for (int q = 0; q < kMfSeg; ++q) {
            const int i = tid + q * kMfThreads;
            const bool in = t0 + i < n;
            const unsigned dst = (unsigned)__cvta_generic_to_shared(P + i);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(in ? row + t0 + i : row),
                         "r"(in ? 4 : 0)
                         : "memory");
        }
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    // exclusive prefix: per-thread segment sums, then a block scan of the totals
    int4 v[kMfSeg / 4];
    int32_t tot = 0;
#pragma unroll
    for (int q = 0; q < kMfSeg / 4; ++q) {
        v[q] = *reinterpret_cast<const int4 *>(P + tid * kMfSeg + 4 * q);
        int32_t e0 = tot, e1 = e0 + v[q].x, e2 = e1 + v[q].y, e3 = e2 + v[q].z;
        tot = e3 + v[q].w;
        v[q] = make_int4(e0, e1, e2, e3);
    }
    int32_t incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    int32_t off = incl - tot;
    for (int w2 = 0; w2 < warp; ++w2) off += s_warp[w2];
#pragma unroll
    for (int q = 0; q < kMfSeg / 4; ++q)
        *reinterpret_cast<int4 *>(P + tid * kMfSeg + 4 * q) =
            make_int4(v[q].x + off, v[q].y + off, v[q].z + off, v[q].w + off);
    __syncthreads();

    int32_t tm[kPows];
#pragma unroll
    for (int j = 0; j < kPows; ++j) tm[j] = s_tmin[j];
    const long long nrem_l = n - t0;  // samples of the row from t0 on
    const int nrem = (int)min((long long)kMfSpan, nrem_l);
    if (tid == 0) tile_sum[(long long)d * ntiles + blockIdx.x] = P[min(kMfTile, nrem)];
    // every cell of the tile and every boxcar lie inside the row
    const bool inside = nrem_l >= (long long)kMfTile + (1 << (31 - __clz(wmask)));
    const long long cbase = (long long)d * n + t0;
#pragma unroll 1
    for (int j = 0; j < kMfTile / (32 * 4 * (kMfThreads / 32)); ++j) {
        const int t = warp * (kMfTile / (kMfThreads / 32)) + j * 128 + lane * 4;  // first of this lane's 4 cells
        const int4 p0 = *reinterpret_cast<const int4 *>(P + t);
        const int2 p45 = *reinterpret_cast<const int2 *>(P + t + 4);
        bool h0 = false, h1 = false, h2 = false, h3 = false;
        if (inside)
            mf_test4<true, ALLW>(P, t, nrem, wmask, tm, p0, p45, h0, h1, h2, h3);
        else
            mf_test4<false, ALLW>(P, t, nrem, wmask, tm, p0, p45, h0, h1, h2, h3);
        const int32_t pc[4] = {p0.x, p0.y, p0.z, p0.w};
        const bool hc[4] = {h0, h1, h2, h3};
        uint32_t nib = 0, live = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const bool lv = t + i < nrem;
            live |= (uint32_t)lv << i;
            nib |= (uint32_t)(lv && hc[i]) << i;
        }
        if (live == 0xFu && ((cbase + t) & 3) == 0) {
            *reinterpret_cast<int4 *>(pre + cbase + t) = p0;  // pre comes from cudaMalloc: 16-byte aligned rows of 4
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if ((live >> i) & 1u) pre[cbase + t + i] = pc[i];
        }
        // cells whose S/N is computed (hot ones, or all with full_map) join
        // the tile's list, warp by warp in cell order
        const uint32_t want = full_map ? live : nib;
        if (__any_sync(0xffffffffu, want != 0u)) {
            const int cnt = __popc(want);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            unsigned wbase = 0;
            if (lane == 31) wbase = atomicAdd(&s_nlist, (unsigned)incl);
            unsigned pos = __shfl_sync(0xffffffffu, wbase, 31) + (unsigned)(incl - cnt);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if ((want >> i) & 1u) s_list[pos++] = (uint16_t)(t + i);
        }
        // eight lanes' nibbles make one 32-cell word of the hot bitmask
        uint32_t word = nib << (4 * (lane & 7));
        word |= __shfl_xor_sync(0xffffffffu, word, 1);
        word |= __shfl_xor_sync(0xffffffffu, word, 2);
        word |= __shfl_xor_sync(0xffffffffu, word, 4);
        const long long tw = t0 + t;  // first cell of the word for lanes 0, 8, 16, 24
        if ((lane & 7) == 0 && tw < n) {
            hotbits[(long long)d * nwr + tw / 32] = word;
            if (word) atomicAdd(&s_nhot, (unsigned)__popc(word));
        }
    }
    __syncthreads();
    if (tid == 0 && s_nhot) atomicAdd(&st->nhot, (unsigned long long)s_nhot);
    // best S/N and width of the listed cells, one cell per thread.  Listed
    // hot cells skip the widths whose sum stays below the threshold sum: their
    // S/N is below the threshold, so below the cell's best (ties included);
    // the full map computes every width
    const unsigned nl = s_nlist;
#pragma unroll 1
    for (unsigned e = tid; e < nl; e += kMfThreads) {
        const int c = s_list[e];
        float bs = 0.0f;
        int bw = 0;
        const int32_t pi = P[c];
#pragma unroll
        for (int j = 0; j < kPows; ++j) {
            const int32_t S = P[c + (1 << j)] - pi;  // inside the staged span: c + 2^j < 4096 + 1024
            if ((ALLW || ((wmask >> j) & 1u)) && c + (1 << j) <= nrem && (full_map || S >= tm[j])) {
                const float snr = ss == 0 ? 0.0f : div_rn((float)S, s_den[j], s_rcp[j]);
                if (bw == 0 || snr > bs) {
                    bs = snr;
                    bw = 1 << j;
                }
            }
        }
        best[cbase + c] = bw ? bs : -INFINITY;  // no width fits before the row end
        bestw[cbase + c] = (uint16_t)bw;
    }
}

// Per row, exclusive prefix of the tile totals: tile_off[d][i] = sum of tiles < i.
__global__ void dd_tile_scan_kernel(const long long *__restrict__ tile_sum, long long *__restrict__ tile_off, int ndm,
                                 int ntiles) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= ndm) return;
    long long acc = 0;
    for (int i = 0; i < ntiles; ++i) {
        tile_off[(long long)d * ntiles + i] = acc;
        acc += tile_sum[(long long)d * ntiles + i];
    }
}

// ---------------------------------------------------------------------------
// grouping: runs of hot cells along time, joined across DM rows
// ---------------------------------------------------------------------------

// hotbits holds, per row, ceil(n/32) words: bit t%32 of word t/32 is set when
// cell (d, t) is hot.  A run is a maximal interval of hot cells in one row and
// its start is the cell where it begins.  The run start of any hot cell
// follows from its word and wl, the last run start before each word: the
// highest run-start bit at or below the cell's bit, else wl of the word.  The
// run starts form a union-find forest in L (entries at run starts only) whose
// roots are the smallest start of each group (deterministic), linked with
// atomicMin.  Two runs in neighbouring rows touch exactly when their
// intervals overlap, and the first column of an overlap is the start of one
// of the two runs, so the rows are joined by visiting only the vertically
// adjacent hot cells that are a run start in either row.
__device__ __forceinline__ uint32_t run_starts(uint32_t m, uint32_t prev_word) {
    return m & ~((m << 1) | (prev_word >> 31));
}

// Run start (cell index) of hot bit b of a word with run-start bits s whose
// bit 0 is cell cw; wl_w = the last run start before the word.
__device__ __forceinline__ int32_t run_start_of(uint32_t s, int b, long long cw, int32_t wl_w) {
    const uint32_t m = s & ((2u << b) - 1u);  // run starts at or below b (b = 31: all)
    return m ? (int32_t)(cw + 31 - __clz(m)) : wl_w;
}

// Per word of row blockIdx.x, the last run start before it (wl), and every
// run start as its own union-find node.  Warp k of the block owns a
// contiguous range of the row's words and walks it 32 words at a time (lane =
// word, coalesced): pass 1 finds the last run start of each range, a scan over
// the warps gives each range the last start before it, and pass 2 writes wl
// from a running max carried across the warp's steps.
__global__ void __launch_bounds__(512) dd_runs_kernel(const uint32_t *__restrict__ hotbits, int nwr, long long n,
                                                      int32_t *__restrict__ L, int32_t *__restrict__ wl) {
    __shared__ int s_warp[16];
    const int d = blockIdx.x;
    const uint32_t *hb = hotbits + (long long)d * nwr;
    const long long cbase = (long long)d * n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per = (nwr + 16 * 32 - 1) / (16 * 32) * 32;  // words per warp, whole steps of 32
    const int w0 = min(nwr, warp * per), w1 = min(nwr, w0 + per);
    // pass 1: last run start (time index) in the warp's range
    int last = -1;
    for (int wb = w0; wb < w1; wb += 32) {
        const int w = wb + lane;
        if (w < w1) {
            const uint32_t s = run_starts(hb[w], w > 0 ? hb[w - 1] : 0u);
            if (s) last = 32 * w + 31 - __clz(s);
        }
    }
    last = __reduce_max_sync(0xffffffffu, last + 1) - 1;  // as unsigned: -1 -> 0
    if (lane == 0) s_warp[warp] = last;
    __syncthreads();
    int carry = -1;
    for (int k = 0; k < warp; ++k) carry = max(carry, s_warp[k]);
    // pass 2
    int32_t *wrow = wl + (long long)d * nwr;
    for (int wb = w0; wb < w1; wb += 32) {
        const int w = wb + lane;
        uint32_t s = 0;
        if (w < w1) s = run_starts(hb[w], w > 0 ? hb[w - 1] : 0u);
        const int lw = s ? 32 * w + 31 - __clz(s) : -1;
        int incl = lw;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl = max(incl, u);
        }
        int before = __shfl_up_sync(0xffffffffu, incl, 1);
        if (lane == 0) before = -1;
        if (w < w1) {
            wrow[w] = (int32_t)(cbase + max(carry, before));  // meaningful when bit 0 continues a run
            for (uint32_t q = s; q; q &= q - 1) {
                const int32_t c = (int32_t)(cbase + 32 * w + __ffs(q) - 1);
                L[c] = c;
            }
        }
        carry = max(carry, __shfl_sync(0xffffffffu, incl, 31));
    }
}

__device__ __forceinline__ int32_t find_root(const int32_t *L, int32_t x) {
    int32_t p = __ldcg(L + x);
    while (p != x) {
        x = p;
        p = __ldcg(L + x);
    }
    return x;
}

// find with path halving: each visited node is pointed at its grandparent.
// Labels only ever move to smaller indices of the same group, so a plain
// store of an ancestor is safe against concurrent links (a linker that loses
// its update sees the changed parent and retries).
__device__ __forceinline__ int32_t find_halving(int32_t *L, int32_t x) {
    int32_t p = __ldcg(L + x);
    while (p != x) {
        const int32_t gp = __ldcg(L + p);
        if (gp != p) __stcg(L + x, gp);
        x = gp;
        p = __ldcg(L + x);
    }
    return x;
}

__device__ void unite(int32_t *L, int32_t a, int32_t b, DevState *st) {
    for (unsigned it = 0; it < kUnionCap; ++it) {
        a = find_halving(L, a);
        b = find_halving(L, b);
        if (a == b) return;
        if (a < b) {
            const int32_t t = a;
            a = b;
            b = t;
        }
        // link the larger root a under b
        const int32_t old = atomicMin(L + a, b);
        if (old == a) return;
        a = old;
    }
    atomicOr(&st->err, 4u);
}

// Join runs of rows d-1 and d that overlap, at the first column of each overlap.
__global__ void dd_vunion_kernel(const uint32_t *__restrict__ hotbits, int nwr, int ndm, long long n, int32_t *L,
                                 const int32_t *__restrict__ wl, DevState *st) {
    // rows on y, words on x: no index division
    for (int d = 1 + blockIdx.y; d < ndm; d += gridDim.y) {
        const uint32_t *h2 = hotbits + (long long)d * nwr, *h1 = h2 - nwr;
        const int32_t *wl2 = wl + (long long)d * nwr, *wl1 = wl2 - nwr;
        for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nwr; w += gridDim.x * blockDim.x) {
            const uint32_t a2 = h2[w], a1 = h1[w];
            const uint32_t v = a1 & a2;
            if (!v) continue;
            const uint32_t s2 = run_starts(a2, w > 0 ? h2[w - 1] : 0u);
            const uint32_t s1 = run_starts(a1, w > 0 ? h1[w - 1] : 0u);
            const long long cw2 = (long long)d * n + 32LL * w;
            for (uint32_t q = v & (s1 | s2); q; q &= q - 1) {
                const int b = __ffs(q) - 1;
                const int32_t a = run_start_of(s2, b, cw2, wl2[w]);
                const int32_t e = run_start_of(s1, b, cw2 - n, wl1[w]);
                unite(L, a, e, st);
            }
        }
    }
}

// Every run start points straight at its root.
__global__ void dd_compress_kernel(const uint32_t *__restrict__ hotbits, int nwr, int ndm, long long n, int32_t *L) {
    for (int d = blockIdx.y; d < ndm; d += gridDim.y) {
        const uint32_t *h = hotbits + (long long)d * nwr;
        for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nwr; w += gridDim.x * blockDim.x) {
            for (uint32_t q = run_starts(h[w], w > 0 ? h[w - 1] : 0u); q; q &= q - 1) {
                const int32_t c = (int32_t)((long long)d * n + 32 * w + __ffs(q) - 1);
                L[c] = find_root(L, c);
            }
        }
    }
}

// Roots get compact ids, stored in place as -(id + 2).
__global__ void dd_ids_kernel(const uint32_t *__restrict__ hotbits, int nwr, int ndm, long long n, int32_t *L,
                              DevState *st) {
    for (int d = blockIdx.y; d < ndm; d += gridDim.y) {
        const uint32_t *h = hotbits + (long long)d * nwr;
        for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nwr; w += gridDim.x * blockDim.x) {
            for (uint32_t q = run_starts(h[w], w > 0 ? h[w - 1] : 0u); q; q &= q - 1) {
                const int32_t c = (int32_t)((long long)d * n + 32 * w + __ffs(q) - 1);
                if (L[c] == c) L[c] = -2 - (int32_t)atomicAdd(&st->nroots, 1u);
            }
        }
    }
}

// Group id of a run start: start -> root (at most two hops after compression).
__device__ __forceinline__ int group_id(const int32_t *L, int32_t start) {
    int32_t v = L[start];
    for (int hop = 0; hop < 2 && v >= 0; ++hop) v = L[v];
    return v <= -2 ? -2 - v : -1;
}

// Per group: the largest (S/N, -cell) key and the number of cells.  A lane
// takes one word; each stretch of consecutive hot bits lies in one run and
// gives one record, and the warp combines records of the same group before
// its atomics.
__global__ void dd_group_reduce_kernel(const uint32_t *__restrict__ hotbits, int nwr, int ndm, long long n,
                                       const int32_t *__restrict__ L, const int32_t *__restrict__ wl,
                                       const float *__restrict__ best, int max_cands,
                                       unsigned long long *__restrict__ key, long long *__restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    // rows on y; a warp takes 32 consecutive words of one row
    for (int d = blockIdx.y; d < ndm; d += gridDim.y)
    for (int w0 = blockIdx.x * blockDim.x + (int)(threadIdx.x & ~31u); w0 < nwr; w0 += gridDim.x * blockDim.x) {
        const int w = w0 + lane;
        const long long k = (long long)d * nwr + w;
        uint32_t q = 0, sq = 0;  // hot bits, run-start bits
        const long long cw = (long long)d * n + 32LL * w;  // cell index of bit 0 of this word
        int32_t wlk = 0;
        if (w < nwr) {
            q = hotbits[k];
            if (q) {
                sq = run_starts(q, w > 0 ? hotbits[k - 1] : 0u);
                wlk = wl[k];
            }
        }
        while (__any_sync(0xffffffffu, q != 0u)) {
            int id = -1;
            unsigned long long kv = 0;
            unsigned cntv = 0;
            if (q) {
                const int b0 = __ffs(q) - 1;
                const uint32_t rest = ~(q >> b0);
                const int len = rest ? __ffs(rest) - 1 : 32 - b0;
                q = len >= 32 - b0 ? 0u : q & ~(((1u << len) - 1u) << b0);
                const int32_t c0 = (int32_t)(cw + b0);
                id = group_id(L, ((sq >> b0) & 1u) ? c0 : wlk);  // a stretch not at a run start begins at bit 0
                if (id >= max_cands) id = -1;
                for (int i = 0; i < len; ++i) {
                    // largest S/N first, then the smallest cell index (lower DM, then earlier time)
                    const uint32_t c = (uint32_t)(c0 + i);
                    const unsigned long long v =
                        ((unsigned long long)__float_as_uint(best[c]) << 32) | (unsigned long long)(0xFFFFFFFFu - c);
                    kv = v > kv ? v : kv;
                }
                cntv = (unsigned)len;
            }
            const unsigned peers = __match_any_sync(0xffffffffu, id);
            unsigned long long m = kv;
            unsigned long long tot = 0;
            for (unsigned p = peers; p; p &= p - 1) {
                const int src = __ffs(p) - 1;
                const unsigned long long v = __shfl_sync(peers, kv, src);
                tot += __shfl_sync(peers, cntv, src);
                m = v > m ? v : m;
            }
            if (id >= 0 && lane == __ffs(peers) - 1) {
                atomicMax(key + id, m);
                atomicAdd(reinterpret_cast<unsigned long long *>(cnt + id), tot);
            }
        }
    }
}

// Mark each group's representative cell in a bitmask, and store its group id
// in the (no longer needed) label array.
__global__ void dd_mark_kernel(const unsigned long long *__restrict__ key, int32_t *__restrict__ L,
                               unsigned *__restrict__ marks, const DevState *st, int max_cands) {
    const int nr = (int)min((unsigned)max_cands, st->nroots);
    for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < nr; id += gridDim.x * blockDim.x) {
        const uint32_t c = 0xFFFFFFFFu - (uint32_t)(key[id] & 0xFFFFFFFFu);
        L[c] = id;
        atomicOr(marks + (c >> 5), 1u << (c & 31));
    }
}

// Ordered compaction of the marked cells (cell order = (DM, time) order):
// per-chunk counts, an exclusive scan over chunks, then an ordered write.  A
// thread owns kCompactWords consecutive words of a chunk.
constexpr int kCompactWords = kCompactChunk / 32 / kCompactThreads;
static_assert(kCompactWords * 32 * kCompactThreads == kCompactChunk, "chunk = threads x words x 32");

__global__ void __launch_bounds__(kCompactThreads) dd_count_marks_kernel(const unsigned *__restrict__ marks,
                                                                         long long nwords,
                                                                         unsigned *__restrict__ chunk_count) {
    __shared__ unsigned s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const long long w0 = (long long)blockIdx.x * (kCompactChunk / 32) + threadIdx.x * kCompactWords;
    unsigned mine = 0;
#pragma unroll
    for (int i = 0; i < kCompactWords; ++i)
        if (w0 + i < nwords) mine += __popc(marks[w0 + i]);
    if (mine) atomicAdd(&s_cnt, mine);
    __syncthreads();
    if (threadIdx.x == 0) chunk_count[blockIdx.x] = s_cnt;
}

__global__ void __launch_bounds__(kCompactThreads) dd_scan_chunks_kernel(unsigned *__restrict__ chunk_count, int nchunks) {
    // single CTA: exclusive scan in place, kCompactThreads entries at a time
    __shared__ unsigned s[kCompactThreads];
    unsigned carry = 0;
    for (int base = 0; base < nchunks; base += kCompactThreads) {
        const int i = base + threadIdx.x;
        const unsigned v = i < nchunks ? chunk_count[i] : 0u;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < kCompactThreads; o <<= 1) {
            const unsigned u = threadIdx.x >= o ? s[threadIdx.x - o] : 0u;
            __syncthreads();
            s[threadIdx.x] += u;
            __syncthreads();
        }
        if (i < nchunks) chunk_count[i] = carry + s[threadIdx.x] - v;
        carry += s[kCompactThreads - 1];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kCompactThreads) dd_write_marks_kernel(
    const unsigned *__restrict__ marks, long long nwords, const uint16_t *__restrict__ bestw,
    const float *__restrict__ best, const int32_t *__restrict__ L, const long long *__restrict__ cnt, long long n,
    int beam, const unsigned *__restrict__ chunk_off, int max_cands, dd_candidate *__restrict__ out) {
    __shared__ unsigned s_warp[kCompactThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long w0 = (long long)blockIdx.x * (kCompactChunk / 32) + threadIdx.x * kCompactWords;
    uint32_t mw[kCompactWords];
    unsigned mine = 0;
#pragma unroll
    for (int i = 0; i < kCompactWords; ++i) {
        mw[i] = w0 + i < nwords ? marks[w0 + i] : 0u;
        mine += __popc(mw[i]);
    }
    // exclusive scan of the threads' counts (thread order = cell order)
    unsigned incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    unsigned pos = chunk_off[blockIdx.x] + incl - mine;
    for (int k = 0; k < warp; ++k) pos += s_warp[k];
#pragma unroll
    for (int i = 0; i < kCompactWords; ++i) {
        for (uint32_t q = mw[i]; q; q &= q - 1) {
            const long long c = (w0 + i) * 32 + __ffs(q) - 1;
            if (pos < (unsigned)max_cands) {
                dd_candidate o;
                o.beam = beam;
                o.d = (int32_t)(c / n);
                o.t = (int32_t)(c % n);
                o.w = bestw[c];
                o.snr = best[c];
                o.score = 0.0f;
                o.ncells = cnt[L[c]];
                out[pos] = o;
            }
            ++pos;
        }
    }
}

// ---------------------------------------------------------------------------
// snippets
// ---------------------------------------------------------------------------

// Row prefix P(t) = sum of y[0..t) from the tile-local prefixes and the tile offsets.
__device__ __forceinline__ long long row_prefix(const int32_t *pre_row, const long long *off_row,
                                                const long long *sum_row, long long n, int ntiles, long long t) {
    if (t <= 0) return 0;
    if (t >= n) return off_row[ntiles - 1] + sum_row[ntiles - 1];
    return off_row[t / kMfTile] + (long long)pre_row[t];
}

__global__ void __launch_bounds__(256) dd_snippet_kernel(const int32_t *__restrict__ pre,
                                                      const long long *__restrict__ tile_off,
                                                      const long long *__restrict__ tile_sum, int ntiles, int ndm,
                                                      long long n, const unsigned long long *__restrict__ sumsq,
                                                      const dd_candidate *__restrict__ cands,
                                                      __nv_bfloat16 *__restrict__ out) {
    __shared__ float s_den[64];  // per snippet row: float(sigma * sqrt(w)), 0 for no data
    const dd_candidate cd = cands[blockIdx.x];
    const int w = cd.w;
    if (threadIdx.x < 64) {
        const int dd = cd.d - 32 + threadIdx.x;
        float den = 0.0f;
        if (dd >= 0 && dd < ndm && sumsq[dd] != 0ULL)
            den = (float)(sqrt((double)sumsq[dd] / (double)n) * sqrt((double)w));
        s_den[threadIdx.x] = den;
    }
    __syncthreads();
    __nv_bfloat16 *o = out + (long long)blockIdx.x * 64 * 64;
    const int lane = threadIdx.x & 31;
    // a warp takes 32 consecutive bins of one row: each lane looks up the
    // prefix at its bin's start and takes its end from the next lane (four
    // rows' lookups in flight at once)
#pragma unroll 4
    for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
        const int r = i >> 6, b = i & 63;
        const int dd = cd.d - 32 + r;
        const float den = s_den[r];  // the same for the whole warp
        float v = 0.0f;
        if (den != 0.0f) {
            const long long s0 = (long long)cd.t + (long long)(b - 32) * w;
            const int32_t *pr = pre + (long long)dd * n;
            const long long *orow = tile_off + (long long)dd * ntiles, *srow = tile_sum + (long long)dd * ntiles;
            const long long p0 = row_prefix(pr, orow, srow, n, ntiles, s0);
            long long p1 = __shfl_down_sync(0xffffffffu, p0, 1);
            if (lane == 31) p1 = row_prefix(pr, orow, srow, n, ntiles, s0 + w);
            v = (float)(p1 - p0) / den;
        }
        o[i] = __float2bfloat16_rn(v);
    }
}

// Snippets straight from y (dd_snippets with caller buffers): each bin sums
// its w samples with warp shuffles.
__global__ void __launch_bounds__(256) dd_snippet_from_y_kernel(const int32_t *__restrict__ y, long long ld_y, int ndm,
                                                      long long n, const unsigned long long *__restrict__ sumsq,
                                                      const dd_candidate *__restrict__ cands,
                                                      __nv_bfloat16 *__restrict__ out) {
    const dd_candidate cd = cands[blockIdx.x];
    const int w = cd.w;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __nv_bfloat16 *o = out + (long long)blockIdx.x * 64 * 64;
    for (int r = warp; r < 64; r += 8) {
        const int dd = cd.d - 32 + r;
        const bool live = dd >= 0 && dd < ndm && sumsq[dd] != 0ULL;
        float den = 1.0f;
        if (live) den = (float)(sqrt((double)sumsq[dd] / (double)n) * sqrt((double)w));
        const int32_t *row = y + (long long)(live ? dd : 0) * ld_y;
        const long long base = (long long)cd.t - 32LL * w;
        // 64 bins of w samples cover [base, base + 64w): read it 32 samples at a time
        long long bin_acc = 0;  // lane 0 keeps the running bin sum when w >= 32
        for (long long s = 0; s < 64LL * w; s += 32) {
            const long long t = base + s + lane;
            long long v = (live && t >= 0 && t < n) ? (long long)row[t] : 0;
            if (w >= 32) {
#pragma unroll
                for (int o2 = 16; o2 > 0; o2 >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o2);
                bin_acc += v;
                if (((s + 32) % w) == 0) {
                    if (lane == 0) {
                        const int b = (int)(s / w);
                        o[r * 64 + b] = __float2bfloat16_rn(live ? (float)bin_acc / den : 0.0f);
                    }
                    bin_acc = 0;
                }
            } else {
                for (int o2 = 1; o2 < w; o2 <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o2);
                if ((lane % w) == 0) {
                    const int b = (int)((s + lane) / w);
                    o[r * 64 + b] = __float2bfloat16_rn(live ? (float)v / den : 0.0f);
                }
            }
        }
    }
}


}  // namespace

struct Search {
    dd_search_config cfg;
    SearchCfgDev dcfg;
    int nbins = 0;
    int32_t *y = nullptr;
    unsigned long long *sumsq = nullptr;
    float *best = nullptr;
    uint16_t *bestw = nullptr;
    int32_t *labels = nullptr;    // union-find forest (entries at run starts only)
    int32_t *wl = nullptr;        // [ndm][ceil(n/32)] last run start before each word
    uint32_t *hotbits = nullptr;  // [ndm][ceil(n/32)] hot-cell bitmask
    unsigned long long *key = nullptr;
    long long *cnt = nullptr;
    dd_candidate *cands = nullptr;
    unsigned *chunk = nullptr;  // per-chunk counts / offsets for the ordered compaction
    int32_t *pre = nullptr;       // tile-local exclusive prefix of y
    unsigned *marks = nullptr;    // representative-cell bitmask
    float *den = nullptr;         // [ndm][nw] S/N denominators
    int32_t *tmin = nullptr;      // [ndm][nw] smallest boxcar sum reaching thresh
    long long *tile_sum = nullptr, *tile_off = nullptr;
    int ntiles = 0;
    size_t nchunks_cap = 0;
    DevState *st = nullptr;
    // last run
    int ndm = 0;
    long long n = 0;
    long long ld_y = 0;
};

static void free_search(Search *s) {
    if (!s) return;
    cudaFree(s->y);
    cudaFree(s->sumsq);
    cudaFree(s->best);
    cudaFree(s->bestw);
    cudaFree(s->labels);
    cudaFree(s->wl);
    cudaFree(s->hotbits);
    cudaFree(s->key);
    cudaFree(s->cnt);
    cudaFree(s->chunk);
    cudaFree(s->pre);
    cudaFree(s->marks);
    cudaFree(s->den);
    cudaFree(s->tmin);
    cudaFree(s->tile_sum);
    cudaFree(s->tile_off);
    cudaFree(s->cands);
    cudaFree(s->st);
    delete s;
}

}  // namespace dd

using namespace dd;

extern "C" {

dd_status dd_search_create(dd_search **out, const dd_search_config *cfg) {
    if (!out || !cfg) return fail(DD_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    const dd_search_config &c = *cfg;
    if (c.ndm_max <= 0 || c.n_max == 0 || c.nchan <= 0 || c.nchan > 21844 || c.half_window <= 0 || c.half_window > 32767 || c.nwidths <= 0 ||
        c.nwidths > kMaxWidths || !(c.thresh > 0) || c.max_cands <= 0 || c.max_cands > DD_SEARCH_MAX_CANDS ||
        c.baseline < 0 || c.baseline > 1)
        return fail(DD_ERR_INVALID_ARG, "bad search configuration");
    if ((double)c.ndm_max * (double)c.n_max >= 2147483647.0)
        return fail(DD_ERR_INVALID_ARG, "ndm_max * n_max must stay below 2^31 (cell indices are int32)");
    for (int k = 0; k < c.nwidths; ++k) {
        const int w = c.widths[k];
        if (w <= 0 || w > 1024 || (w & (w - 1)) || (k > 0 && w <= c.widths[k - 1]))
            return fail(DD_ERR_INVALID_ARG, "widths must be ascending powers of two <= 1024");
    }
    Search *s = new (std::nothrow) Search();
    if (!s) return fail(DD_ERR_NOMEM, "host allocation failed");
    s->cfg = c;
    s->dcfg.nw = c.nwidths;
    for (int k = 0; k < kMaxWidths; ++k) s->dcfg.widths[k] = k < c.nwidths ? c.widths[k] : 0;
    s->dcfg.wmask = 0;
    for (int k = 0; k < c.nwidths; ++k) s->dcfg.wmask |= (unsigned)c.widths[k];
    s->nbins = 3 * c.nchan + 1;
    const size_t cells = (size_t)c.ndm_max * c.n_max;
    cudaError_t e = cudaMalloc(&s->y, cells * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s->sumsq, (size_t)c.ndm_max * 8);
    if (e == cudaSuccess) e = cudaMalloc(&s->best, cells * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s->bestw, cells * 2);
    if (e == cudaSuccess) e = cudaMalloc(&s->labels, cells * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s->hotbits, (size_t)c.ndm_max * ((c.n_max + 31) / 32) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s->wl, (size_t)c.ndm_max * ((c.n_max + 31) / 32) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s->key, (size_t)c.max_cands * 8);
    if (e == cudaSuccess) e = cudaMalloc(&s->cnt, (size_t)c.max_cands * 8);
    if (e == cudaSuccess) e = cudaMalloc(&s->cands, (size_t)c.max_cands * sizeof(dd_candidate));
    s->nchunks_cap = (cells + kCompactChunk - 1) / kCompactChunk;
    if (e == cudaSuccess) e = cudaMalloc(&s->chunk, s->nchunks_cap * sizeof(unsigned));
    const size_t tiles_cap = (size_t)c.ndm_max * ((c.n_max + kMfTile - 1) / kMfTile);
    if (e == cudaSuccess) e = cudaMalloc(&s->pre, cells * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s->marks, (cells + 31) / 32 * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s->den, (size_t)c.ndm_max * kMaxWidths * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s->tmin, (size_t)c.ndm_max * kMaxWidths * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s->tile_sum, tiles_cap * 8);
    if (e == cudaSuccess) e = cudaMalloc(&s->tile_off, tiles_cap * 8);
    if (e == cudaSuccess) e = cudaMalloc(&s->st, sizeof(DevState));
    if (e == cudaSuccess) e = cudaMemset(s->st, 0, sizeof(DevState));
    if (e != cudaSuccess) {
        dd_status st = cuda_fail(e, "allocating search buffers");
        free_search(s);
        return st;
    }
    *out = reinterpret_cast<dd_search *>(s);
    return DD_OK;
}

dd_status dd_search_run(dd_search *search, const uint32_t *d_x, size_t ld_x, int ndm, size_t n, int beam,
                        void *stream) {
    Search *s = reinterpret_cast<Search *>(search);
    if (!s || !d_x) return fail(DD_ERR_INVALID_ARG, "NULL search or input");
    if (ndm <= 0 || ndm > s->cfg.ndm_max || n == 0 || n > s->cfg.n_max || ld_x < n)
        return fail(DD_ERR_INVALID_ARG, "ndm/n beyond the search capacity or ld_x < n");
    cudaStream_t st = (cudaStream_t)stream;
    s->ndm = ndm;
    s->n = (long long)n;
    s->ld_y = (long long)n;
    DD_CUDA_TRY(cudaMemsetAsync(s->sumsq, 0, (size_t)ndm * 8, st));
    DD_CUDA_TRY(cudaMemsetAsync(s->st, 0, sizeof(DevState), st));
    DD_CUDA_TRY(cudaMemsetAsync(s->key, 0, (size_t)s->cfg.max_cands * 8, st));
    DD_CUDA_TRY(cudaMemsetAsync(s->cnt, 0, (size_t)s->cfg.max_cands * 8, st));
    // baseline
    const long long h = s->cfg.half_window;
    s->ntiles = (int)((n + kMfTile - 1) / kMfTile);
    if (s->cfg.baseline == 1 && mean_fused_smem(h) <= kMeanFusedSmemMax) {
        const size_t sm = mean_fused_smem(h);
        static thread_local size_t configured = 0;
        if (sm > 48 * 1024 && sm > configured) {
            DD_CUDA_TRY(cudaFuncSetAttribute(dd_mean_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            configured = sm;
        }
        dd_mean_fused_kernel<<<dim3((unsigned)(((long long)n + kMeanTile - 1) / kMeanTile), (unsigned)ndm), kMeanThreads,
                               sm, st>>>(d_x, (long long)ld_x, (long long)n, h, (uint32_t)(s->nbins - 1), s->y, s->ld_y,
                                         s->sumsq, s->st);
    } else if (s->cfg.baseline == 1) {
        dd_xprefix_kernel<<<dim3((unsigned)s->ntiles, (unsigned)ndm), 256, 0, st>>>(
            d_x, (long long)ld_x, (long long)n, (uint32_t)(s->nbins - 1), s->pre, s->tile_sum, s->ntiles, s->st);
        dd_tile_scan_kernel<<<(ndm + 127) / 128, 128, 0, st>>>(s->tile_sum, s->tile_off, ndm, s->ntiles);
        dd_mean_apply_kernel<<<dim3((unsigned)(((long long)n + kMeanCells - 1) / kMeanCells), (unsigned)ndm), 256, 0,
                               st>>>(
            d_x, (long long)ld_x, (long long)n, h, (uint32_t)(s->nbins - 1), s->pre, s->tile_off, s->tile_sum,
            s->ntiles, s->y, s->ld_y, s->sumsq);
    } else {
        const long long nsegs = (long long)ndm * (((long long)n + h - 1) / h);
        const unsigned grid = (unsigned)((nsegs + 31) / 32);
        if (s->nbins - 1 > 32767)  // outputs need more than 16 bits
            dd_median_kernel<true><<<grid, 32, med_smem_bytes<true>(), st>>>(
                d_x, (long long)ld_x, ndm, (long long)n, (int)h, s->nbins, s->y, s->ld_y, s->sumsq, s->st);
        else
            dd_median_kernel<false><<<grid, 32, med_smem_bytes<false>(), st>>>(
                d_x, (long long)ld_x, ndm, (long long)n, (int)h, s->nbins, s->y, s->ld_y, s->sumsq, s->st);
    }
    DD_CUDA_TRY(cudaGetLastError());
    // matched filter + sigma cut
    dim3 fg((unsigned)((n + kMfTile - 1) / kMfTile), (unsigned)ndm);
    s->ntiles = (int)((n + kMfTile - 1) / kMfTile);
    dd_thresh_kernel<<<(ndm * s->cfg.nwidths + 127) / 128, 128, 0, st>>>(s->sumsq, (long long)n, s->dcfg,
                                                                        s->cfg.thresh, ndm, s->den, s->tmin);
    const int nwr = (int)((n + 31) / 32);
    if (s->dcfg.wmask == (1u << kPows) - 1u)
        dd_mf_kernel<true><<<fg, kMfThreads, 0, st>>>(s->y, s->ld_y, (long long)n, s->sumsq, s->dcfg, s->cfg.thresh, s->best,
                                             s->bestw, s->hotbits, nwr, s->st, s->pre, s->tile_sum, s->ntiles, s->den,
                                             s->tmin, s->cfg.full_map);
    else
        dd_mf_kernel<false><<<fg, kMfThreads, 0, st>>>(s->y, s->ld_y, (long long)n, s->sumsq, s->dcfg, s->cfg.thresh, s->best,
                                             s->bestw, s->hotbits, nwr, s->st, s->pre, s->tile_sum, s->ntiles, s->den,
                                             s->tmin, s->cfg.full_map);
    DD_CUDA_TRY(cudaGetLastError());
    dd_tile_scan_kernel<<<(ndm + 127) / 128, 128, 0, st>>>(s->tile_sum, s->tile_off, ndm, s->ntiles);
    // grouping
    const int g = 152 * 8;
    const long long cells = (long long)ndm * (long long)n;
    dd_runs_kernel<<<ndm, 512, 0, st>>>(s->hotbits, nwr, (long long)n, s->labels, s->wl);
    // word kernels: words of a row on x, rows on y
    const dim3 gw((unsigned)std::min((nwr + 255) / 256, 64), (unsigned)std::min(ndm, 4096));
    dd_vunion_kernel<<<gw, 256, 0, st>>>(s->hotbits, nwr, ndm, (long long)n, s->labels, s->wl, s->st);
    dd_compress_kernel<<<gw, 256, 0, st>>>(s->hotbits, nwr, ndm, (long long)n, s->labels);
    dd_ids_kernel<<<gw, 256, 0, st>>>(s->hotbits, nwr, ndm, (long long)n, s->labels, s->st);
    dd_group_reduce_kernel<<<gw, 256, 0, st>>>(s->hotbits, nwr, ndm, (long long)n, s->labels, s->wl, s->best,
                                              s->cfg.max_cands, s->key, s->cnt);
    const long long nwords = (cells + 31) / 32;
    DD_CUDA_TRY(cudaMemsetAsync(s->marks, 0, (size_t)nwords * 4, st));
    dd_mark_kernel<<<g, 256, 0, st>>>(s->key, s->labels, s->marks, s->st, s->cfg.max_cands);
    const int nchunks = (int)((cells + kCompactChunk - 1) / kCompactChunk);
    dd_count_marks_kernel<<<nchunks, kCompactThreads, 0, st>>>(s->marks, nwords, s->chunk);
    dd_scan_chunks_kernel<<<1, kCompactThreads, 0, st>>>(s->chunk, nchunks);
    dd_write_marks_kernel<<<nchunks, kCompactThreads, 0, st>>>(s->marks, nwords, s->bestw, s->best, s->labels, s->cnt,
                                                               (long long)n, beam, s->chunk, s->cfg.max_cands,
                                                               s->cands);
    return cuda_fail(cudaGetLastError(), "search kernels");
}

}  // extern "C"

namespace dd {
const unsigned *search_dev_ngroups(const dd_search *search) {
    return &reinterpret_cast<const Search *>(search)->st->nroots;
}
}  // namespace dd

extern "C" {

dd_status dd_search_result(const dd_search *search, long long *nhot, int *ngroups, unsigned *flags, void *stream) {
    const Search *s = reinterpret_cast<const Search *>(search);
    if (!s) return fail(DD_ERR_INVALID_ARG, "NULL search");
    DevState h;
    DD_CUDA_TRY(cudaMemcpyAsync(&h, s->st, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    DD_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    if (nhot) *nhot = (long long)h.nhot;
    if (ngroups) *ngroups = (int)h.nroots;
    if (flags) *flags = h.err;
    return DD_OK;
}

dd_status dd_search_stats(const dd_search *search, long long *median_rebuilds, void *stream) {
    const Search *s = reinterpret_cast<const Search *>(search);
    if (!s) return fail(DD_ERR_INVALID_ARG, "NULL search");
    DevState h;
    DD_CUDA_TRY(cudaMemcpyAsync(&h, s->st, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    DD_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    if (median_rebuilds) *median_rebuilds = (long long)h.nrebuild;
    return DD_OK;
}

dd_status dd_search_candidates(const dd_search *search, dd_candidate *host_out, int max, int *count, void *stream) {
    const Search *s = reinterpret_cast<const Search *>(search);
    if (!s || !count) return fail(DD_ERR_INVALID_ARG, "NULL search or count");
    int ng = 0;
    dd_status r = dd_search_result(search, nullptr, &ng, nullptr, stream);
    if (r != DD_OK) return r;
    const int avail = std::min(ng, s->cfg.max_cands);
    *count = avail;
    const int k = std::min(avail, max);
    if (k > 0 && host_out) {
        DD_CUDA_TRY(cudaMemcpyAsync(host_out, s->cands, (size_t)k * sizeof(dd_candidate), cudaMemcpyDeviceToHost,
                                    (cudaStream_t)stream));
        DD_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    }
    return DD_OK;
}

dd_status dd_search_device_candidates(const dd_search *search, const dd_candidate **d_cands) {
    const Search *s = reinterpret_cast<const Search *>(search);
    if (!s || !d_cands) return fail(DD_ERR_INVALID_ARG, "NULL argument");
    *d_cands = s->cands;
    return DD_OK;
}

dd_status dd_search_buffers(const dd_search *search, const int32_t **d_y, const int64_t **d_sumsq,
                            const float **d_best, const uint16_t **d_bestw) {
    const Search *s = reinterpret_cast<const Search *>(search);
    if (!s) return fail(DD_ERR_INVALID_ARG, "NULL search");
    if (d_y) *d_y = s->y;
    if (d_sumsq) *d_sumsq = reinterpret_cast<const int64_t *>(s->sumsq);
    if (d_best) *d_best = s->best;
    if (d_bestw) *d_bestw = s->bestw;
    return DD_OK;
}

dd_status dd_snippets(const int32_t *d_y, size_t ld_y, int ndm, size_t n, const int64_t *d_sumsq, int ncand,
                      const dd_candidate *d_cands, uint16_t *d_out, void *stream) {
    if (!d_y || !d_sumsq || !d_cands || !d_out || ndm <= 0 || n == 0 || ld_y < n || ncand < 0)
        return fail(DD_ERR_INVALID_ARG, "bad snippet arguments");
    if (ncand == 0) return DD_OK;
    dd_snippet_from_y_kernel<<<ncand, 256, 0, (cudaStream_t)stream>>>(
        d_y, (long long)ld_y, ndm, (long long)n, reinterpret_cast<const unsigned long long *>(d_sumsq), d_cands,
        reinterpret_cast<__nv_bfloat16 *>(d_out));
    return cuda_fail(cudaGetLastError(), "dd_snippet_kernel launch");
}

dd_status dd_search_snippets(const dd_search *search, int ncand, uint16_t *d_out, void *stream) {
    const Search *s = reinterpret_cast<const Search *>(search);
    if (!s || !d_out || ncand < 0) return fail(DD_ERR_INVALID_ARG, "NULL search or output");
    if (ncand > s->cfg.max_cands) return fail(DD_ERR_INVALID_ARG, "ncand beyond the candidate capacity");
    if (ncand == 0) return DD_OK;
    dd_snippet_kernel<<<ncand, 256, 0, (cudaStream_t)stream>>>(s->pre, s->tile_off, s->tile_sum, s->ntiles, s->ndm,
                                                            s->n, s->sumsq, s->cands,
                                                            reinterpret_cast<__nv_bfloat16 *>(d_out));
    return cuda_fail(cudaGetLastError(), "dd_snippet_kernel launch");
}

void dd_search_destroy(dd_search *search) { free_search(reinterpret_cast<Search *>(search)); }

}  // extern "C"
