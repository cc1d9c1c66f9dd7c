// Device code of the tiled dedispersion kernel, shared by the single-gulp
// launch and the persistent multi-beam launch.  See dedisp_kernels.cu for the
// method; this header holds the tile routine and its helpers.
#pragma once

#include "dd_internal.h"
#include "tc.cuh"

namespace dd {
namespace tiled {

constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;
constexpr int kGroup = 64;  // default channels per shared-memory stage (one carry-save tree)

// log2 of a stage's channel count G (32, 64 or 128): the depth of its tree.
template <int G>
struct GroupLog {
    static_assert(G == 32 || G == 64 || G == 128, "channel stage of 32, 64 or 128");
    static constexpr int value = G == 32 ? 5 : (G == 64 ? 6 : 7);
};

struct TiledArgs {
    const uint32_t *in;     // packed input as 32-bit words (16 samples each)
    long long ld_w;         // words per channel row
    const uint32_t *tab;    // [n_dmb][nchan][D]: (slot word address << 5) | funnel shift, per (channel, trial)
    const int32_t *wsrel;   // [n_dmb][nchan]: first staged word of the channel, relative to the tile
    int nchan;
    int ndm;
    long long nout;
    uint32_t *out;
    long long ld_out;
    int slot;   // shared-memory words per staged channel
    int n_dmb;  // DM blocks
    unsigned *err;        // device error word: bit 0 when a tile gave up waiting for its staged input
    uint32_t poll_limit;  // polls of a stage's mbarrier before the tile gives up (kStagePollLimit)
};

// Polls of a stage's mbarrier before a tile gives up on its input.  A poll
// that finds the phase incomplete suspends the thread for a few microseconds
// (about 2.5 us measured on GB300), so this is some 40 ms: far beyond the
// microseconds a stage copy takes, and short enough that a launch whose
// copies never land still ends within seconds.
constexpr uint32_t kStagePollLimit = 1u << 14;

// Words of one shared-memory stage: G channel slots plus a zero slot,
// rounded up to 4 words so the 16-byte table copies after the stages stay aligned.
__host__ __device__ constexpr int tile_stage_words(int slot, int G = kGroup) { return ((G + 1) * slot + 3) / 4 * 4; }

// Staged words per channel for W words per lane and a DM block whose delays
// spread over `spread` samples: the 32*W lane words, the next word for the
// funnel shift, the spread, and up to 3 words that start the window on a
// 16-byte boundary, rounded up to whole 16-byte groups.
inline int tile_slot(int W, int spread) { return (32 * W + (spread + 15) / 16 + 4 + 3) / 4 * 4; }

// Shared-memory layout of a tile, in 32-bit words: the two stages'
// mbarriers (4 words, at the same place for every plan, so a persistent CTA
// keeps them across beams), two stages of windows, two [G][D] tables, then
// the nchan window bases.
constexpr int kBarWords = 4;
__host__ __device__ constexpr size_t tile_smem_bytes(int slot, int G, int D, int nchan) {
    return (size_t)(kBarWords + 2 * tile_stage_words(slot, G) + 2 * G * D + nchan) * 4;
}

// Host side: the tables of DM blocks of D trials (tab [n_dmb][nchan_pad][D],
// nchan_pad = nchan rounded up to the stage's G channels; wsrel
// [n_dmb][nchan]) from the delay table [ndm][nchan].  wsrel is the
// first staged word of a channel relative to the time tile, rounded down to a
// multiple of 4 words (the tile's first word is one too); a table entry is
// (byte offset of the trial's first word in the stage << 5) | (2 * sample
// offset within that word).  Padded channels point at the stage's zero slot.
inline void build_tile_tables(const int32_t *delays, int ndm, int nchan, int D, int slot, uint32_t *tab,
                              int32_t *wsrel, int G = kGroup) {
    const int n_dmb = (ndm + D - 1) / D;
    const int nchan_pad = (nchan + G - 1) / G * G;
    const uint32_t zero_slot = (uint32_t)(4 * G * slot) << 5;
    for (int b = 0; b < n_dmb; ++b) {
        const int d0 = b * D;
        for (int c = 0; c < nchan_pad; ++c) {
            uint32_t *row = tab + ((size_t)b * nchan_pad + c) * D;
            if (c >= nchan) {
                for (int j = 0; j < D; ++j) row[j] = zero_slot;
                continue;
            }
            const int32_t dl0 = delays[(size_t)d0 * nchan + c];
            const int32_t r = (dl0 >> 4) & 3;  // words between the aligned window start and the first trial's word
            wsrel[(size_t)b * nchan + c] = (dl0 >> 4) - r;
            const int cl = c % G;
            for (int j = 0; j < D; ++j) {
                const int d = d0 + j < ndm ? d0 + j : ndm - 1;
                const int32_t o = (dl0 & 15) + delays[(size_t)d * nchan + c] - dl0;
                const uint32_t byte_off = (uint32_t)(4 * (cl * slot + r + (o >> 4)));
                row[j] = (byte_off << 5) | (uint32_t)(2 * (o & 15));
            }
        }
    }
}

// One 3-input logic op on 32 bit positions (truth table lut over inputs a, b, c).
template <unsigned lut>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(lut));
    return d;
}

// Full adder on 32 independent bit positions: sum (a xor b xor c, table 0x96)
// and carry (majority, table 0xE8) of a+b+c, one logic op each.
__device__ __forceinline__ void full_add(uint32_t &carry, uint32_t &sum, uint32_t a, uint32_t b, uint32_t c) {
    sum = lop3<0x96>(a, b, c);
    carry = lop3<0xE8>(a, b, c);
}

template <int DT, int W>
struct Ctx {
    const char *win;      // this lane's view of the stage: stage base + 4*lane bytes
    const uint32_t *tab;  // [G][D] packed (byte offset, shift)
    int jbase;            // first trial of this warp within the CTA
};

// Which output words a lane owns: with an odd W > 1, W consecutive words
// (lane*W ..), so the W+1 staged words they need are read once each, with a
// lane stride of W words that is free of bank conflicts; otherwise the words
// lane, lane+32, ...
template <int W>
struct LaneWords {
    static constexpr bool contiguous = (W % 2 == 1) && W > 1;
    static __device__ __forceinline__ int first(int lane) { return contiguous ? lane * W : lane; }
    static __device__ __forceinline__ int word(int lane, int i) { return contiguous ? lane * W + i : lane + 32 * i; }
};

// 16 samples of channel c realigned to trial jj's delay, for each of the
// lane's W words: one funnel shift of two consecutive staged words.  A table
// entry is (byte offset in the stage << 5) | shift; the funnel shift only
// reads the low 5 bits.  Channels past the band's end point at a zero slot.
template <int DT, int W>
__device__ __forceinline__ void fetch(const Ctx<DT, W> &x, int c, uint32_t (&v)[DT][W]) {
    constexpr int D = kWarps * DT;
#pragma unroll
    for (int jj = 0; jj < DT; ++jj) {
        const uint32_t e = x.tab[c * D + x.jbase + jj];
        const uint32_t *p = reinterpret_cast<const uint32_t *>(x.win + (e >> 5));
        if constexpr (LaneWords<W>::contiguous) {
            uint32_t r[W + 1];
#pragma unroll
            for (int i = 0; i <= W; ++i) r[i] = p[i];
#pragma unroll
            for (int i = 0; i < W; ++i) v[jj][i] = __funnelshift_r(r[i], r[i + 1], e);
        } else {
#pragma unroll
            for (int i = 0; i < W; ++i) v[jj][i] = __funnelshift_r(p[32 * i], p[32 * i + 1], e);
        }
    }
}

// Harley-Seal carry-save tree: add channels [cb, cb + 2^L) into bit-planes
// P[0..L-1] (bit k of plane P[k] counts 2^k); returns the carry of weight 2^L.
template <int L, int DT, int W, int NP>
__device__ __forceinline__ void hs(const Ctx<DT, W> &x, uint32_t (&P)[DT][W][NP], uint32_t (&carry)[DT][W], int cb) {
    if constexpr (L == 1) {
        uint32_t a[DT][W], b[DT][W];
        fetch(x, cb, a);
        fetch(x, cb + 1, b);
#pragma unroll
        for (int jj = 0; jj < DT; ++jj)
#pragma unroll
            for (int i = 0; i < W; ++i) full_add(carry[jj][i], P[jj][i][0], P[jj][i][0], a[jj][i], b[jj][i]);
    } else {
        uint32_t ca[DT][W], cc[DT][W];
        hs<L - 1>(x, P, ca, cb);
        hs<L - 1>(x, P, cc, cb + (1 << (L - 1)));
#pragma unroll
        for (int jj = 0; jj < DT; ++jj)
#pragma unroll
            for (int i = 0; i < W; ++i)
                full_add(carry[jj][i], P[jj][i][L - 1], P[jj][i][L - 1], ca[jj][i], cc[jj][i]);
    }
}

// Minimum resident CTAs per SM the register budget is sized for.
template <int DT, int W, int NP>
struct TileOcc {
    static constexpr int value = (DT * W * NP > 66) ? 1 : 2;
};

// Once per CTA, before its first tile: one arrival per stage copy (G window
// rows and the table) on each stage's mbarrier.  The caller synchronises the
// block before the first tile.
template <int G>
__device__ __forceinline__ void tile_init_bars(uint32_t *smem) {
    if (threadIdx.x == 0) {
        uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
        tc::mbar_init(&bars[0], G + 1);
        tc::mbar_init(&bars[1], G + 1);
        tc::fence_mbar_init();
    }
}

// One output tile: DM block dmb (D = 8*DT trials) x time tile tt (512*W
// samples), the band taken G channels per shared-memory stage.  smem holds
// tile_smem_bytes() with its mbarriers initialised by tile_init_bars; bit b
// of `phase` is the parity of stage buffer b's next completion and carries
// over to the CTA's next tile.  Returns false (in every thread) when a stage
// never arrived within the poll limit; the tile's outputs are then not
// written and the error word has bit 0 set.  The caller synchronises the
// block before reusing the shared memory.
template <int DT, int W, int NP, int G>
__device__ __forceinline__ bool dd_tile(const TiledArgs &a, int dmb, long long tt, uint32_t *smem, uint32_t &phase) {
    constexpr int D = kWarps * DT;
    constexpr int TW = 32 * W;
    constexpr long long T = 16LL * TW;
    constexpr int LG = GroupLog<G>::value;
    static_assert(NP > LG, "more bit-planes than the tree's depth");
    // the stages' mbarriers, two stages of [G+1][slot] windows (the last
    // slot stays zero and stands in for channels past the band's end), then
    // two [G][D] tables, then the channel bases
    const int stage_words = tile_stage_words(a.slot, G);
    uint64_t *const s_bar = reinterpret_cast<uint64_t *>(smem);
    uint32_t *const s_win0 = smem + kBarWords;
    uint32_t *const s_tab0 = s_win0 + 2 * stage_words;
    int32_t *s_ws = reinterpret_cast<int32_t *>(s_win0 + 2 * stage_words + 2 * G * D);

    const int d0 = dmb * D;
    const long long t0 = tt * T;
    const long long tw0 = t0 >> 4;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int nchan_pad = (a.nchan + G - 1) / G * G;
    const uint32_t *gtab = a.tab + (long long)dmb * nchan_pad * D;
    const int32_t *gws = a.wsrel + (long long)dmb * a.nchan;
    const int nchunks = (a.nchan + G - 1) / G;

    for (int c = threadIdx.x; c < a.nchan; c += kThreads) s_ws[c] = __ldg(gws + c);
    for (int w = threadIdx.x; w < a.slot; w += kThreads) {
        s_win0[G * a.slot + w] = 0u;
        s_win0[stage_words + G * a.slot + w] = 0u;
    }
    __syncthreads();

    // copy one stage with the copy engine: thread cl < G moves channel cl's
    // packed window in one bulk copy (the window start, the time tile's first
    // word, the row stride and the slot are all multiples of 4 words, so
    // addresses and sizes are multiples of 16 bytes), thread G the stage's
    // (address, shift) table rows; each adds its bytes to the stage
    // mbarrier's transaction count before copying.  A window is cut at the
    // row's end: words past it only ever feed outputs beyond nout.
    auto stage = [&](int k, int b) {
        const int c0 = k * G;
        const int t = threadIdx.x;
        if (t < G) {
            uint32_t bytes = 0;
            long long ws = 0;
            if (c0 + t < a.nchan) {
                ws = tw0 + s_ws[c0 + t];
                const long long nw = min((long long)a.slot, a.ld_w - ws);
                bytes = nw > 0 ? (uint32_t)(4 * nw) : 0u;
            }
            tc::mbar_arrive_expect_tx(&s_bar[b], bytes);
            if (bytes)
                tc::bulk_copy_g2s(s_win0 + b * stage_words + t * a.slot, a.in + (long long)(c0 + t) * a.ld_w + ws,
                                  bytes, &s_bar[b]);
        } else if (t == G) {
            const uint32_t bytes = (uint32_t)(4 * G * D);
            tc::mbar_arrive_expect_tx(&s_bar[b], bytes);
            tc::bulk_copy_g2s(s_tab0 + b * (G * D), gtab + (long long)c0 * D, bytes, &s_bar[b]);
        }
    };

    uint32_t P[DT][W][NP];
#pragma unroll
    for (int jj = 0; jj < DT; ++jj)
#pragma unroll
        for (int i = 0; i < W; ++i)
#pragma unroll
            for (int k = 0; k < NP; ++k) P[jj][i][k] = 0u;

    bool ok = true;
    stage(0, 0);
    for (int k = 0; k < nchunks; ++k) {
        if (k + 1 < nchunks) stage(k + 1, (k + 1) & 1);
        // stage k is in once its mbarrier completes the phase of this use
        const int b = k & 1;
        if (ok) ok = tc::mbar_wait(&s_bar[b], (phase >> b) & 1u, a.poll_limit);
        phase ^= 1u << b;
        Ctx<DT, W> x{reinterpret_cast<const char *>(s_win0 + (k & 1) * stage_words + LaneWords<W>::first(lane)),
                     s_tab0 + (k & 1) * (G * D), warp * DT};
        uint32_t cg[DT][W];
        hs<LG>(x, P, cg, 0);
        // ripple the weight-G carry into the upper planes
#pragma unroll
        for (int jj = 0; jj < DT; ++jj)
#pragma unroll
            for (int i = 0; i < W; ++i) {
                uint32_t c = cg[jj][i];
#pragma unroll
                for (int l = LG; l < NP; ++l) {
                    const uint32_t s = P[jj][i][l] ^ c;
                    c &= P[jj][i][l];
                    P[jj][i][l] = s;
                }
            }
        __syncthreads();
    }
    if (__syncthreads_or(!ok)) {
        // a stage never arrived: record it, give both buffers' last copies
        // one more short bounded wait, and leave the outputs alone
        if (threadIdx.x == 0) atomicOr(a.err, 1u);
        const uint32_t last = a.poll_limit / 64 + 1;
        for (int b = 0; b < 2; ++b) tc::mbar_wait(&s_bar[b], ((phase >> b) & 1u) ^ 1u, last);
        return false;
    }

    // bit-planes -> per-sample sums.  2-bit lane r of a plane holds (low bit,
    // high bit) of sample r; masking lanes r and r+8 into 16-bit halves gives
    // sum_k 2^k * lane = count(low) + 2*count(high) <= 3*nchan < 65536.
#pragma unroll
    for (int jj = 0; jj < DT; ++jj) {
        const int d = d0 + warp * DT + jj;
        if (d >= a.ndm) continue;
        uint32_t *orow = a.out + (long long)d * a.ld_out;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const long long t = t0 + 16LL * LaneWords<W>::word(lane, i);
            if (t >= a.nout) continue;
            uint32_t v[16];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                uint32_t h = 0u;
#pragma unroll
                for (int k = 0; k < NP; ++k) h += ((P[jj][i][k] >> (2 * r)) & 0x00030003u) << k;
                v[r] = h & 0xFFFFu;
                v[r + 8] = h >> 16;
            }
            if (t + 16 <= a.nout) {
                uint4 *o4 = reinterpret_cast<uint4 *>(orow + t);
#pragma unroll
                for (int q = 0; q < 4; ++q) o4[q] = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            } else {
#pragma unroll
                for (int m = 0; m < 16; ++m)
                    if (t + m < a.nout) orow[t + m] = v[m];
            }
        }
    }
    return true;
}

// Work list of the persistent multi-beam kernel: tile_start[b] is the first
// global tile index of beam b (tiles of a beam are DM block fastest).
struct BatchDesc {
    int nbeams;
    int pad;
    long long ntiles;
    long long tile_start[DD_BATCH_MAX_BEAMS + 1];
    TiledArgs beam[DD_BATCH_MAX_BEAMS];
};

}  // namespace tiled
}  // namespace dd
