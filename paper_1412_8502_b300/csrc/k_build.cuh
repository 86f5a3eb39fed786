// Pair-list rebuild (the cell-list build of Sec. II.B.2, re-designed for the
// GPU): a counting sort of the particles over a Hilbert-ordered grid of
// 2^(3 nbits) bins per species, a deterministic in-bin order, 32-particle
// tiles with FP64 origins and bounding boxes, and per-tile lists of the
// tiles whose bounding boxes come within the interaction range plus skin.
//
// Rebuild rule (the neighbour-list rule of Sec. II.B.1 applied to tiles):
// rebuild when any particle has moved more than skin/2 - (L - L_build)
// since the last rebuild, or every `rebuild_every` steps.  A particle that
// crossed a face after the rebuild re-enters shifted by the box growth
// since its crossing (Eq. 3 grows L, positions are not rescaled), so in its
// tile's frame it has moved by at most its displacement plus L - L_build.
// Every pair closer than the cutoff now was then closer than cutoff + skin
// at the rebuild, so its tiles' boxes were within cutoff + skin.
#include "kernels.h"

namespace pasta {

namespace {

// Hilbert index of the bin (qx, qy, qz) of a 2^nbits grid: Skilling's
// transpose method ("Programming the Hilbert curve", AIP Conf. Proc. 707,
// 2004) -- undo the excess work of the Gray-code inverse level by level,
// Gray-encode, then interleave the bits with axis x most significant.
// Consecutive indices are face-adjacent bins, so a run of 32 particles in
// this order occupies a compact region.
__device__ inline unsigned hilbert_key(unsigned qx, unsigned qy, unsigned qz, int nbits) {
    unsigned X[3] = {qx, qy, qz};
    const unsigned M = 1u << (nbits - 1);
    for (unsigned Q = M; Q > 1; Q >>= 1) {
        const unsigned P = Q - 1;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;
            } else {
                const unsigned t = (X[0] ^ X[i]) & P;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    unsigned t = 0;
    for (unsigned Q = M; Q > 1; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1;
    X[0] ^= t;
    X[1] ^= t;
    X[2] ^= t;
    unsigned h = 0;
    for (int k = nbits - 1; k >= 0; --k)
        h = (h << 3) | (((X[0] >> k) & 1u) << 2) | (((X[1] >> k) & 1u) << 1) | ((X[2] >> k) & 1u);
    return h;
}

// Bin of a position in [0, L): FP32 arithmetic on the truncated position (a
// bin choice near a bin face is as good as the other; every later step uses
// the stored key).
__device__ inline unsigned sort_key(const SysConst& S, double x, double y, double z, double L) {
    const int n = 1 << S.nbits;
    const float sc = (float)n / narrow_trunc(L);
    const int qx = min(max((int)(narrow_trunc(x) * sc), 0), n - 1);
    const int qy = min(max((int)(narrow_trunc(y) * sc), 0), n - 1);
    const int qz = min(max((int)(narrow_trunc(z) * sc), 0), n - 1);
    return hilbert_key((unsigned)qx, (unsigned)qy, (unsigned)qz, S.nbits);
}

// Inclusive scan over a block of 1024 threads; returns the exclusive prefix
// of v and writes the block total to *total.
__device__ inline unsigned block_exscan(unsigned v, unsigned* sm /*32*/, unsigned* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) sm[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        unsigned s = lane < nw ? sm[lane] : 0u;
        unsigned si = s;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += y;
        }
        if (lane < nw) sm[lane] = si - s;
        if (lane == 31) sm[32] = si;
    }
    __syncthreads();
    unsigned r = sm[w] + inc - v;
    if (total) *total = sm[32];
    __syncthreads();
    return r;
}

__device__ inline bool sys_rebuilds(const SysConst& S) { return S.st->rebuild != 0; }

// Order-preserving integer keys: a < b exactly when key(a) < key(b).
__device__ __forceinline__ unsigned long long dkey(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_inv(unsigned long long k) {
    const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

// Bounds lo <= min and hi >= max of v over the valid lanes of the warp from
// one 32-bit integer reduction each on the high words of the keys (no FP64
// arithmetic): the bounds are the doubles at the ends of the high-word
// intervals, within 2^-20 of the true extremes relative to their magnitude.
// At least one lane must be valid.
__device__ __forceinline__ void warp_bounds(double v, bool valid, double& lo, double& hi) {
    const unsigned k = (unsigned)(dkey(v) >> 32);
    const unsigned kmin = __reduce_min_sync(0xffffffffu, valid ? k : 0xffffffffu);
    const unsigned kmax = __reduce_max_sync(0xffffffffu, valid ? k : 0u);
    lo = dkey_inv((unsigned long long)kmin << 32);
    hi = dkey_inv(((unsigned long long)kmax << 32) | 0xffffffffull);
}

}  // namespace

// ---------------------------------------------------------------- decision
// One thread per system.  forced_only: rebuild only systems that asked.
// set_cond: the kernel runs inside a step graph whose rebuild kernels sit in
// two conditional (IF) nodes, on handles cond_cell and cond_list (a handle
// drives one node); it sets both, so the rebuild kernels are not launched at
// all on steps without a rebuild.
__device__ __forceinline__ void decide_body(const EngineDev& E, int forced_only, int only,
                                            cudaGraphConditionalHandle cond_cell, cudaGraphConditionalHandle cond_list,
                                            int set_cond, cudaGraphConditionalHandle cond_var, int set_var) {
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    for (int s = threadIdx.x; s < E.nsys; s += blockDim.x) {
        const SysConst& S = E.sys[s];
        SysState* st = S.st;
        int need = st->force_rebuild;
        if (!forced_only) {
            const float md2 = __uint_as_float(st->maxdisp2);
            const float h = (float)(0.5 * S.skin - (st->L - st->L_build));
            need |= (st->step - st->last_build >= S.rebuild_every) || (h <= 0.0f) || (md2 > h * h);
        }
        if (only >= 0 && s != only) need = 0;
        // energy record of this step's force pass (step graphs launch no
        // separate clear)
        for (int k = 0; k < 6; ++k) st->eacc[k] = 0;
        st->maxdisp2 = 0u;
        st->rebuild = need;
        st->cur_next = need ? (st->cur ^ 1) : st->cur;
        if (need) {
            st->force_rebuild = 0;
            st->hmax = 0u;
            st->hsum = 0.0f;
            st->list_total = 0;
            st->vtop = 0ull;
            st->vpairs = 0ull;
            atomicOr(&any, 1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *E.any_rebuild = any;
        if (set_cond) {
            cudaGraphSetConditional(cond_cell, any ? 1u : 0u);
            cudaGraphSetConditional(cond_list, any ? 1u : 0u);
            if (any) *E.cond_runs += 1ull;
        }
        // force-pass code variant of this step: fixed by system 0's
        // force_unroll, else the tuner's
        ForceTune* tu = E.tune;
        const int fu = E.nsys > 0 ? E.sys[0].force_unroll : 0;
        const int sel = fu == 4 ? 0 : fu == 2 ? 1 : fu == 1 ? 2 : fu == 3 ? 3 : tu->cur;
        tu->sel = sel;
        if (set_var) cudaGraphSetConditional(cond_var, (unsigned)sel);
    }
}

__global__ void k_decide(EngineDev E, int forced_only, int only, cudaGraphConditionalHandle cond_cell,
                         cudaGraphConditionalHandle cond_list, int set_cond, cudaGraphConditionalHandle cond_var,
                         int set_var) {
    griddep_wait();
    decide_body(E, forced_only, only, cond_cell, cond_list, set_cond, cond_var, set_var);
}

// ---------------------------------------------------------------- histogram
// Bins of kScanChunk consecutive global bins form the chunks of the bin scan.
constexpr int kScanPer = 8;
constexpr int kScanChunk = 1024 * kScanPer;

// Key and bin count of every particle of a rebuilding system.
__device__ __forceinline__ void hist_body(const EngineDev& E, int bx) {
    if (!*E.any_rebuild) return;
    const int g = bx * kTilesPerBlock + (threadIdx.x >> 5);
    if (g >= E.ntiles) return;
    const int s = E.tile_sys[g];
    if (s < 0) return;
    const SysConst& S = E.sys[s];
    if (!sys_rebuilds(S)) return;
    const int t = g - S.tile_base;
    if (t >= S.T) return;
    const int p = tile_slot0(S, t) + (threadIdx.x & 31);
    if (p >= tile_end(S, t)) return;
    const SysState* st = S.st;
    const double* x = S.x[st->cur];
    const unsigned k = sort_key(S, x[p], x[S.N + p], x[2 * S.N + p], st->L) +
                       (p < S.Np ? 0u : (unsigned)S.nbins);
    S.key[p] = k;
    atomicAdd(&E.hist[S.bin_base + k], 1u);
}

__global__ void k_hist(EngineDev E) {
    griddep_wait();
    hist_body(E, blockIdx.x);
}

// ---------------------------------------------------------------- bin scan
// Exclusive scan of hist over all systems' bins in two passes: the count of
// each chunk of kScanChunk bins (k_scan_reduce), then each chunk scanned by a
// block of 1024 threads from the sum of the counts of the chunks before it
// (k_scan_bins).  Exact integer sums: the result is that of any other order
// of summation.

static_assert(kScanPer == 8, "a thread's bins are two 16-byte vectors");

// The 8 bins of a thread from base: two 16-byte loads (bases are multiples
// of 8 bins; the allocation is 256-byte aligned), element loads at the tail.
__device__ __forceinline__ void load8(const unsigned* a, long long base, long long n, unsigned (&v)[kScanPer]) {
    if (base + kScanPer <= n) {
        const uint4 p = *reinterpret_cast<const uint4*>(a + base);
        const uint4 q = *reinterpret_cast<const uint4*>(a + base + 4);
        v[0] = p.x; v[1] = p.y; v[2] = p.z; v[3] = p.w;
        v[4] = q.x; v[5] = q.y; v[6] = q.z; v[7] = q.w;
    } else {
        for (int k = 0; k < kScanPer; ++k) v[k] = (base + k < n) ? a[base + k] : 0u;
    }
}
__device__ __forceinline__ void store8(unsigned* a, long long base, long long n, const unsigned (&v)[kScanPer]) {
    if (base + kScanPer <= n) {
        *reinterpret_cast<uint4*>(a + base) = make_uint4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<uint4*>(a + base + 4) = make_uint4(v[4], v[5], v[6], v[7]);
    } else {
        for (int k = 0; k < kScanPer; ++k)
            if (base + k < n) a[base + k] = v[k];
    }
}

__global__ void k_scan_reduce(EngineDev E) {
    griddep_wait();
    if (!*E.any_rebuild) return;
    __shared__ unsigned sm[33];
    const long long base = (long long)blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
    unsigned v[kScanPer];
    load8(E.hist, base, E.nbins_total, v);
    unsigned s = 0;
    for (int k = 0; k < kScanPer; ++k) s += v[k];
    unsigned tot;
    block_exscan(s, sm, &tot);
    if (threadIdx.x == 0) E.blocksum[blockIdx.x] = tot;
}

// Sum of the chunk counts before chunk vb, in every thread of the block.
__device__ __forceinline__ unsigned chunk_offset(const EngineDev& E, int vb, unsigned* sm) {
    unsigned o = 0;
    for (int c = threadIdx.x; c < vb; c += blockDim.x) o += E.blocksum[c];
    unsigned tot;
    block_exscan(o, sm, &tot);
    return tot;
}

__global__ void k_scan_bins(EngineDev E) {
    griddep_wait();
    if (!*E.any_rebuild) return;
    __shared__ unsigned sm[33];
    const unsigned off = chunk_offset(E, blockIdx.x, sm);
    const long long base = (long long)blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
    unsigned v[kScanPer];
    load8(E.hist, base, E.nbins_total, v);
    unsigned s = 0;
    for (int k = 0; k < kScanPer; ++k) s += v[k];
    unsigned run = block_exscan(s, sm, nullptr) + off;
    unsigned o[kScanPer];
    for (int k = 0; k < kScanPer; ++k) {
        o[k] = run;
        run += v[k];
    }
    store8(E.binstart, base, E.nbins_total, o);
    store8(E.cursor, base, E.nbins_total, o);
}

// ---------------------------------------------------------------- scatter
// Places each slot index in its bin (order inside a bin decided by atomics,
// fixed up deterministically by k_move).
__device__ __forceinline__ void scatter_body(const EngineDev& E, int bx) {
    if (!*E.any_rebuild) return;
    const int g = bx * kTilesPerBlock + (threadIdx.x >> 5);
    if (g >= E.ntiles) return;
    const int s = E.tile_sys[g];
    if (s < 0) return;
    const SysConst& S = E.sys[s];
    if (!sys_rebuilds(S)) return;
    const int t = g - S.tile_base;
    if (t >= S.T) return;
    const int p = tile_slot0(S, t) + (threadIdx.x & 31);
    if (p >= tile_end(S, t)) return;
    const unsigned base = E.binstart[S.bin_base];
    const unsigned pos = atomicAdd(&E.cursor[S.bin_base + S.key[p]], 1u) - base;
    S.slot[pos] = p;
}

__global__ void k_scatter(EngineDev E) {
    griddep_wait();
    scatter_body(E, blockIdx.x);
}

// Destination of slot q's particle: its bin start plus the number of
// particles of the same bin with a smaller previous slot index (stable,
// deterministic).  Moves x, v, id (the forces are evaluated after the
// rebuild, or placed by id when a state is loaded with its forces).
__device__ __forceinline__ void move_body(const EngineDev& E, int bx) {
    if (!*E.any_rebuild) return;
    const int g = bx * kTilesPerBlock + (threadIdx.x >> 5);
    if (g >= E.ntiles) return;
    const int s = E.tile_sys[g];
    if (s < 0) return;
    const SysConst& S = E.sys[s];
    if (!sys_rebuilds(S)) return;
    const int t = g - S.tile_base;
    if (t >= S.T) return;
    const int q = tile_slot0(S, t) + (threadIdx.x & 31);
    if (q >= tile_end(S, t)) return;
    const SysState* st = S.st;
    const int c = st->cur, cn = st->cur_next;
    const int j = S.slot[q];
    const unsigned gb = (unsigned)S.key[j];
    const unsigned base = E.binstart[S.bin_base];
    const int s0 = (int)(E.binstart[S.bin_base + gb] - base);
    const int n = (int)E.hist[S.bin_base + gb];
    int rank = 0;
    for (int k = 0; k < n; ++k) rank += (S.slot[s0 + k] < j);
    const int d = s0 + rank;
    const int N = S.N;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        S.x[cn][a * N + d] = S.x[c][a * N + j];
        S.v[cn][a * N + d] = S.v[c][a * N + j];
    }
    S.id[cn][d] = S.id[c][j];
}

__global__ void k_move(EngineDev E) {
    griddep_wait();
    move_body(E, blockIdx.x);
}

// ---------------------------------------------------------------- tiles
// Warp per tile: bounding box, FP64 origin (box centre), FP32 local
// coordinates, displacement reset.  Also clears the system's histogram for
// the next rebuild and records the rebuild.
__device__ __forceinline__ void tiles_body(const EngineDev& E, int bx) {
    if (!*E.any_rebuild) return;
    const int g = bx * kTilesPerBlock + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= E.ntiles) return;
    const int s = E.tile_sys[g];
    if (s < 0) return;
    const SysConst& S = E.sys[s];
    if (!sys_rebuilds(S)) return;
    const int t = g - S.tile_base;
    SysState* st = S.st;
    // clear this system's bins (grid-stride over the system's threads)
    {
        const long long nb = 2 * S.nbins;
        const long long tid = (long long)(g - S.tile_base) * kTile + lane;
        const long long nthr = (long long)((S.T + kTilesPerBlock - 1) / kTilesPerBlock) * kBlock;
        for (long long b = tid; b < nb; b += nthr) E.hist[S.bin_base + b] = 0u;
    }
    __shared__ float s_hm[kTilesPerBlock], s_hs[kTilesPerBlock];
    const int w = threadIdx.x >> 5;
    if (lane == 0) {
        s_hm[w] = 0.0f;
        s_hs[w] = 0.0f;
    }
    if (t < S.T) {
    const int p0 = tile_slot0(S, t), p1 = tile_end(S, t);
    const int p = p0 + lane;
    const bool valid = p < p1;
    const int cn = st->cur_next;
    const int N = S.N;
    const double* x = S.x[cn];
    // FP32 box from the FP64 bounds: the lower bound truncated (positions are
    // >= 0), the upper one truncated and stepped one unit up; no FP64
    // arithmetic (FP64 instructions occupy the narrow FP64 unit even with
    // one active lane).  FP32 rounding of the centre and half extents
    // (< 1e-4 fm below 2000 fm) is covered by the list build's margin.
    float c[3], h[3];
    double xv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        xv[a] = valid ? x[a * N + p] : 0.0;
        double lo, hi;
        warp_bounds(xv[a], valid, lo, hi);
        const float lf = narrow_trunc(lo);
        const float hf = __uint_as_float(__float_as_uint(narrow_trunc(hi)) + 1u);
        c[a] = 0.5f * (lf + hf);
        h[a] = 0.5f * (hf - lf);
    }
    const double L = st->L;
    // The box is that of the wrapped positions themselves (a Hilbert run of
    // [0, L)^3 does not wrap), so every position is within h <= L/2 of the
    // origin and is its own image nearest the origin.
    store_xt(S, t, lane, xv, valid);
    if (valid) {
        S.disp[p] = 0.0f;
        S.disp[N + p] = 0.0f;
        S.disp[2 * N + p] = 0.0f;
    }
    if (lane == 0) {
        const float hm = fmaxf(h[0], fmaxf(h[1], h[2]));
        for (int a = 0; a < 3; ++a) {
            // round the FP32 box up so the FP32 range test stays conservative
            S.thalf[3 * t + a] = h[a] * (1.0f + 1e-6f) + 1e-6f;
            S.torgf[4 * t + a] = c[a];
        }
        S.torgf[4 * t + 3] = hm;
        s_hm[w] = hm;
        s_hs[w] = (h[0] + h[1] + h[2]) * (1.0f / 3.0f);
        if (t == 0) {
            st->last_build = st->step;
            st->n_rebuilds += 1;
            st->L_build = L;
        }
    }
    }
    // one atomic per block for the system's largest / summed half-extents
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.0f, sum = 0.0f;
        for (int k = 0; k < kTilesPerBlock; ++k) {
            m = fmaxf(m, s_hm[k]);
            sum += s_hs[k];
        }
        atomic_max_pos(&st->hmax, m);
        atomicAdd(&st->hsum, sum);
    }
}

__global__ void k_tiles(EngineDev E) {
    griddep_wait();
    tiles_body(E, blockIdx.x);
}

// ---------------------------------------------------------------- lists
// FP32 test "bounding boxes of I and J (nearest image) closer than R".
// Rounding of the FP32 origins (< 1e-4 fm for L < 2000 fm) is covered by
// the margin kMargin, so the test can only include extra tiles.
constexpr float kMargin = 2e-3f;

struct ListTest {
    float Lf, iLf;
    float R2same, R2cross;     // squared ranges: same-species / cross-species
    float R2nuc;               // squared nuclear range (flag for p-p entries)
    int cluster;               // 1: cluster lists (J only proton tiles)
};

__device__ inline ListTest make_test(const SysConst& S, int mode, float L) {
    ListTest T;
    T.Lf = L;
    T.iLf = 1.0f / L;
    if (mode == 0) {
        const float rn = (float)(S.r_nuc + S.skin) + kMargin;
        const float rc = (float)((S.coulomb == 1 ? fmax(S.r_C, S.r_nuc) : S.r_nuc) + S.skin) + kMargin;
        T.R2same = rc * rc;      // used for proton-proton only, see below
        T.R2cross = rn * rn;
        T.R2nuc = rn * rn;
        T.cluster = 0;
    } else {
        // boxes are those of the last rebuild: every particle has drifted
        // by at most skin/2 since then
        const float rpp = (float)(S.r_pp + S.skin) + kMargin, rnp = (float)(S.r_np + S.skin) + kMargin;
        T.R2same = rpp * rpp;
        T.R2cross = rnp * rnp;
        T.R2nuc = 0.0f;
        T.cluster = 1;
    }
    return T;
}

// Squared distance between the FP32 boxes of tiles I and J (nearest image).
__device__ inline float box_d2(const SysConst& S, const float4& oI, const float* hI, int J,
                               const ListTest& T) {
    const float4 oJ = *reinterpret_cast<const float4*>(&S.torgf[4 * J]);
    float d2 = 0.0f;
    float dd[3] = {oI.x - oJ.x, oI.y - oJ.y, oI.z - oJ.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float d = dd[a];
        d -= T.Lf * rintf(d * T.iLf);
        float gap = fabsf(d) - (hI[a] + S.thalf[3 * J + a]);   // symmetric in I and J
        gap = fmaxf(gap, 0.0f);
        d2 = fmaf(gap, gap, d2);
    }
    return d2;
}

// Entry for J from I, or -1 if out of range (see kJMask / kShiftPos /
// kNucBit).  The shift moves J's frame next to I's: s = rint((O_I - O_J)/L).
__device__ inline int list_entry(const SysConst& S, int I, int J, const float4& oI, const float* hI,
                                 const ListTest& T) {
    const bool Ip = I < S.Tp, Jp = J < S.Tp;
    if (T.cluster && !Jp) return -1;
    const float d2 = box_d2(S, oI, hI, J, T);
    int e;
    if (T.cluster) {
        if (!(d2 < (Ip ? T.R2same : T.R2cross))) return -1;
        return J;
    }
    if (Ip && Jp) {
        if (!(d2 < T.R2same)) return -1;
        e = J | (d2 < T.R2nuc ? kNucBit : 0);
    } else {
        if (!(d2 < T.R2cross)) return -1;
        e = J | kNucBit;
    }
    const float4 oJ = *reinterpret_cast<const float4*>(&S.torgf[4 * J]);
    const int sx = (int)rintf((oI.x - oJ.x) * T.iLf);
    const int sy = (int)rintf((oI.y - oJ.y) * T.iLf);
    const int sz = (int)rintf((oI.z - oJ.z) * T.iLf);
    return e | (((sx + 1) | ((sy + 1) << 2) | ((sz + 1) << 4)) << kShiftPos);
}

// Boxes of super-tiles (32 consecutive tiles, compact in Hilbert order):
// one warp each, lane k taking member tile 32 s + k; the union of the member
// boxes from exact integer min / max reductions of the FP32 box faces.
__device__ __forceinline__ void super_body(const EngineDev& E, int bx) {
    if (!*E.any_rebuild) return;
    const int g = bx * kTilesPerBlock + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= E.ntiles) return;
    const int s = E.tile_sys[g];
    if (s < 0) return;
    const SysConst& S = E.sys[s];
    if (!sys_rebuilds(S)) return;
    const int I = g - S.tile_base;           // one warp per tile; the warp of every 32nd tile works
    if (I >= S.T || (I % kTile) != 0) return;
    const int t = I + lane;
    const bool member = t < S.T;
    float lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float c = member ? S.torgf[4 * t + a] : 0.0f, h = member ? S.thalf[3 * t + a] : 0.0f;
        lo[a] = fkey_inv(__reduce_min_sync(0xffffffffu, member ? fkey(c - h) : 0xffffffffu));
        hi[a] = fkey_inv(__reduce_max_sync(0xffffffffu, member ? fkey(c + h) : 0u));
    }
    if (lane != 0) return;
    // half extents rounded up, as for tiles
    S.sorg[I / kTile] = make_float4(0.5f * (lo[0] + hi[0]), 0.5f * (lo[1] + hi[1]), 0.5f * (lo[2] + hi[2]), 0.f);
    S.shalf[I / kTile] = make_float4(0.5f * (hi[0] - lo[0]) * (1.0f + 1e-6f) + 1e-4f,
                                     0.5f * (hi[1] - lo[1]) * (1.0f + 1e-6f) + 1e-4f,
                                     0.5f * (hi[2] - lo[2]) * (1.0f + 1e-6f) + 1e-4f, 0.f);
}

__global__ void k_super(EngineDev E) {
    griddep_wait();
    super_body(E, blockIdx.x);
}

// Force lists in one pass: tile I's entries go to list[I*T ...], its count
// to lcount[I] (the list buffer holds T entries per tile, the worst case).
// Super-tiles out of range of I (widest range) are skipped whole.
// half = 1 (split precision): every unordered tile pair is listed once, the
// forces of each pair being applied to both particles.  The pair {I, J} goes
// to I when (I < J) differs from the parity of I + J, so that every tile
// owns about half of its neighbours wherever it sits in the Hilbert order;
// the tile itself is left out (the force kernel treats it first).
// half = 0 (FP64 validation): full lists, the tile itself included.
__device__ __forceinline__ bool owns_pair(int I, int J, int half) {
    if (!half) return true;
    return J != I && ((I < J) != (((I + J) & 1) != 0));
}

__device__ __forceinline__ void lbuild_body(const EngineDev& E, int half, int bx) {
    if (!*E.any_rebuild) return;
    const int g = bx * kTilesPerBlock + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= E.ntiles) return;
    const int s = E.tile_sys[g];
    if (s < 0) return;
    const SysConst& S = E.sys[s];
    SysState* st = S.st;
    if (!sys_rebuilds(S)) return;
    const int I = g - S.tile_base;
    if (I == 0 && lane == 0) {
        st->cur = st->cur_next;
        // small boxes: tiles are too large for one image per tile pair
        const float hm = __uint_as_float(st->hmax);
        const double rmax = (S.coulomb == 1 ? fmax(S.r_C, S.r_nuc) : S.r_nuc);
        st->need_wrap = (rmax + S.skin + 2.0 * (double)hm + 1e-3 >= 0.5 * st->L) ? 1 : 0;
    }
    if (I >= S.T) return;
    const ListTest T = make_test(S, 0, (float)st->L);
    const float4 oI = *reinterpret_cast<const float4*>(&S.torgf[4 * I]);
    const float hI[3] = {S.thalf[3 * I], S.thalf[3 * I + 1], S.thalf[3 * I + 2]};
    int* lst = S.list + (long long)I * S.T;
    int out = 0, outf = 0;         // near entries from the front, Coulomb-only from the back
    const int nsup = (S.T + kTile - 1) / kTile;
    const bool Ip = I < S.Tp;
    const bool paired = half && S.list_kind == 0;
    for (int s0 = 0; s0 < nsup; s0 += 32) {
        const int sg = s0 + lane;
        bool pass = false;
        if (sg < nsup) {
            const float4 c = S.sorg[sg], h = S.shalf[sg];
            const float dd[3] = {oI.x - c.x, oI.y - c.y, oI.z - c.z};
            const float hh[3] = {h.x, h.y, h.z};
            float d2 = 0.0f;
            for (int a = 0; a < 3; ++a) {
                float d = dd[a];
                d -= T.Lf * rintf(d * T.iLf);
                const float gap = fmaxf(fabsf(d) - hI[a] - hh[a], 0.0f);
                d2 = fmaf(gap, gap, d2);
            }
            // proton-proton pairs reach to the Coulomb range, all others to
            // the nuclear range (super-tiles hold proton tiles first)
            pass = d2 < ((Ip && sg * kTile < S.Tp) ? T.R2same : T.R2cross);
        }
        unsigned sm = __ballot_sync(0xffffffffu, pass);
        while (sm) {
            int J;
            if (paired) {
                // Half lists: of two consecutive tiles 2m, 2m + 1 I owns at
                // most one, so a lane takes the owned tile of a pair and the
                // warp covers two super-tiles (half-warps) per round.
                const int b0 = __ffs(sm) - 1;
                sm &= sm - 1;
                const int b1 = sm ? __ffs(sm) - 1 : -1;
                if (b1 >= 0) sm &= sm - 1;
                const int b = (lane < 16) ? b0 : b1;
                J = -1;
                if (b >= 0) {
                    const int Ja = (s0 + b) * kTile + 2 * (lane & 15);
                    if (Ja < S.T && owns_pair(I, Ja, 1)) J = Ja;
                    else if (Ja + 1 < S.T && owns_pair(I, Ja + 1, 1)) J = Ja + 1;
                }
            } else {
                const int b = __ffs(sm) - 1;
                sm &= sm - 1;
                J = (s0 + b) * kTile + lane;
                if (J >= S.T) J = -1;
            }
            const int e = J >= 0 ? list_entry(S, I, J, oI, hI, T) : -1;
            const bool near = e >= 0 && (e & kNucBit);
            const unsigned mn = __ballot_sync(0xffffffffu, near);
            const unsigned mf = __ballot_sync(0xffffffffu, e >= 0 && !near);
            const unsigned below = (1u << lane) - 1u;
            if (near) lst[out + __popc(mn & below)] = e;
            else if (e >= 0) lst[S.T - 1 - (outf + __popc(mf & below))] = e;
            out += __popc(mn);
            outf += __popc(mf);
        }
    }
    if (lane == 0) {
        S.lcount[I] = out + outf;
        S.lnear[I] = out;
        atomicAdd((unsigned long long*)&st->list_total, (unsigned long long)(out + outf));
    }
}

__global__ void k_lbuild(EngineDev E, int half) {
    griddep_wait();
    lbuild_body(E, half, blockIdx.x);
}

// Per-particle Verlet lists (list_kind 1), built from the full tile-pair
// lists: one block of kVB warps per tile I; lane l keeps every particle j of
// the listed tiles (I itself included, l excluded) with |x_l - x_j| <
// cutoff + skin, the Coulomb cutoff for proton pairs when the Coulomb term
// is on.  Warp w takes list entries w, w + kVB, ...; pass 1 counts, the
// counts are prefixed over the warps (warp order), the tile takes
// 32 x (largest lane total) pool slots, and pass 2 writes each warp's part
// at its offset.  An entry is the source's tile slot 32 J + k, the tile
// pair's periodic shift code and kNucBit when the pair lies inside the
// nuclear range + skin (its low parts are then needed).  A tile that finds
// the pool exhausted keeps an empty list and raises error bit 2.
constexpr int kVB = 4;

__global__ void __launch_bounds__(kVB * 32) k_vbuild(EngineDev E) {
    griddep_wait();
    __shared__ float4 sh[kVB][kTile], sl[kVB][kTile];
    __shared__ int cnts[kVB][kTile];
    __shared__ long long s_base;
    __shared__ int s_width;
    if (!*E.any_rebuild) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x;
    if (g >= E.ntiles) return;
    const int s = E.tile_sys[g];
    if (s < 0) return;
    const SysConst& S = E.sys[s];
    if (S.list_kind != 1 || !sys_rebuilds(S)) return;
    const int I = g - S.tile_base;
    if (I >= S.T) return;
    SysState* st = S.st;
    const double L = st->L;
    const float Lhi = __double2float_rn(L), Llo = __double2float_rn(L - (double)Lhi), iLf = 1.0f / Lhi;
    const bool wrap = st->need_wrap != 0;
    const int nv = tile_end(S, I) - tile_slot0(S, I);
    const bool valid = lane < nv;
    const float4 hi = S.xhi[I * kTile + lane], lo = S.xlo[I * kTile + lane];
    const bool Ip = I < S.Tp;
    const float rn = (float)(S.r_nuc + S.skin) + kMargin;
    const float rc = (float)((S.coulomb == 1 ? fmax(S.r_C, S.r_nuc) : S.r_nuc) + S.skin) + kMargin;
    const float R2n = rn * rn, R2c = rc * rc;
    const int* lst = S.list + (long long)I * S.T;
    const int nl = S.lcount[I], nnear = S.lnear[I];
    long long base = 0;
    int cnt = 0;
    for (int pass = 0; pass < 2; ++pass) {
        for (int e = w; e < nl; e += kVB) {
            const int ent = lst[list_pos(S, e, nnear)];
            const int J = ent & kJMask;
            const int shk = (ent >> kShiftPos) & 63;
            float4 h = S.xhi[J * kTile + lane], l = S.xlo[J * kTile + lane];
            if (shk != kShiftNone) apply_shift(shk, Lhi, Llo, h, l);
            __syncwarp();
            sh[w][lane] = h;
            sl[w][lane] = l;
            __syncwarp();
            const float R2 = (Ip && J < S.Tp) ? R2c : R2n;
            const int nJ = tile_end(S, J) - tile_slot0(S, J);
            for (int k = 0; k < nJ; ++k) {
                const float4 q = sh[w][k], u = sl[w][k];
                float dx = (hi.x - q.x) + (lo.x - u.x);
                float dy = (hi.y - q.y) + (lo.y - u.y);
                float dz = (hi.z - q.z) + (lo.z - u.z);
                if (wrap) {
                    const float kx = rintf(dx * iLf), ky = rintf(dy * iLf), kz = rintf(dz * iLf);
                    dx = fmaf(-Llo, kx, fmaf(-Lhi, kx, dx));
                    dy = fmaf(-Llo, ky, fmaf(-Lhi, ky, dy));
                    dz = fmaf(-Llo, kz, fmaf(-Lhi, kz, dz));
                }
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                if (valid && r2 < R2 && !(J == I && k == lane)) {
                    if (pass == 1)
                        S.vlist[base + 32ll * cnt + lane] =
                            (J * kTile + k) | (shk << kShiftPos) | (r2 < R2n ? kNucBit : 0);
                    ++cnt;
                }
            }
        }
        if (pass == 0) {
            cnts[w][lane] = cnt;
            __syncthreads();
            int off = 0, tot = 0;
            for (int q = 0; q < kVB; ++q) {
                if (q < w) off += cnts[q][lane];
                tot += cnts[q][lane];
            }
            if (w == 0) {
                const int width = (int)__reduce_max_sync(0xffffffffu, (unsigned)tot);
                if (lane == 0) {
                    const unsigned long long b = atomicAdd(&st->vtop, 32ull * (unsigned long long)width);
                    s_base = (long long)b;
                    s_width = width;
                    if ((long long)b + 32ll * width > S.vcap) {
                        atomicOr(&st->error, 4);
                        s_width = -1;
                    }
                }
            }
            __syncthreads();
            if (s_width < 0) {                      // pool exhausted: empty list
                if (w == 0) S.vcount[I * kTile + lane] = 0;
                if (threadIdx.x == 0) {
                    S.voff[I] = 0;
                    S.vwidth[I] = 0;
                }
                return;
            }
            base = s_base;
            cnt = off;                              // this warp writes after the lower warps
            if (w == 0) S.vcount[I * kTile + lane] = tot;
        }
    }
    if (threadIdx.x == 0) {
        S.voff[I] = s_base;
        S.vwidth[I] = s_width;
    }
    if (w == 0) {
        int tot = 0;
        for (int q = 0; q < kVB; ++q) tot += cnts[q][lane];
        const unsigned all = __reduce_add_sync(0xffffffffu, (unsigned)tot);
        if (lane == 0) atomicAdd(&st->vpairs, (unsigned long long)all);
    }
}

// Cluster lists: count, scan, write into a buffer sized by the host.  Boxes
// are those of the last rebuild; the cluster ranges add the skin.
// Proton tiles J in cluster range of tile I, in ascending order: proton
// super-tiles (32 consecutive tiles) out of range of I are skipped whole,
// then the members of the others are tested (visit(J) for each hit).
template <typename Visit>
__device__ __forceinline__ void cluster_tiles(const SysConst& S, int I, int lane, const ListTest& T,
                                              const float4& oI, const float* hI, Visit&& visit) {
    const float R2 = (I < S.Tp) ? T.R2same : T.R2cross;
    const int nsp = (S.Tp + kTile - 1) / kTile;          // super-tiles holding proton tiles
    for (int s0 = 0; s0 < nsp; s0 += 32) {
        const int sg = s0 + lane;
        bool pass = false;
        if (sg < nsp) {
            const float4 c = S.sorg[sg], h = S.shalf[sg];
            const float dd[3] = {oI.x - c.x, oI.y - c.y, oI.z - c.z};
            const float hh[3] = {h.x, h.y, h.z};
            float d2 = 0.0f;
            for (int a = 0; a < 3; ++a) {
                float d = dd[a];
                d -= T.Lf * rintf(d * T.iLf);
                const float gap = fmaxf(fabsf(d) - hI[a] - hh[a], 0.0f);
                d2 = fmaf(gap, gap, d2);
            }
            pass = d2 < R2;
        }
        unsigned sm = __ballot_sync(0xffffffffu, pass);
        while (sm) {
            const int b = __ffs(sm) - 1;
            sm &= sm - 1;
            const int J = (s0 + b) * kTile + lane;
            const int e = J < S.Tp ? list_entry(S, I, J, oI, hI, T) : -1;
            visit(e);
        }
    }
}

__global__ void k_lcount(EngineDev E, int only) {
    const int g = blockIdx.x * kTilesPerBlock + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= E.ntiles) return;
    const int s = E.tile_sys[g];
    if (s < 0 || (only >= 0 && s != only)) return;
    const SysConst& S = E.sys[s];
    SysState* st = S.st;
    const int I = g - S.tile_base;
    if (I >= S.T) return;
    const ListTest T = make_test(S, 1, (float)st->L);
    const float4 oI = *reinterpret_cast<const float4*>(&S.torgf[4 * I]);
    const float hI[3] = {S.thalf[3 * I], S.thalf[3 * I + 1], S.thalf[3 * I + 2]};
    int cnt = 0;
    cluster_tiles(S, I, lane, T, oI, hI, [&](int e) { cnt += __popc(__ballot_sync(0xffffffffu, e >= 0)); });
    if (lane == 0) S.cl->count[I] = cnt;
}

// One block per system: exclusive scan of the tile counts.
__global__ void k_lscan(EngineDev E, int only) {
    const int s = blockIdx.x;
    if (only >= 0 && s != only) return;
    const SysConst& S = E.sys[s];
    __shared__ unsigned sm[33];
    const int* cnt = S.cl->count;
    int* start = S.cl->start;
    const int per = (S.T + blockDim.x - 1) / blockDim.x;
    const int t0 = threadIdx.x * per;
    unsigned sum = 0;
    for (int k = 0; k < per; ++k)
        if (t0 + k < S.T) sum += (unsigned)cnt[t0 + k];
    unsigned tot;
    unsigned run = block_exscan(sum, sm, &tot);
    for (int k = 0; k < per; ++k)
        if (t0 + k < S.T) {
            start[t0 + k] = (int)run;
            run += (unsigned)cnt[t0 + k];
        }
    if (threadIdx.x == 0) {
        start[S.T] = (int)tot;
        *S.cl->total = tot;
    }
}

__global__ void k_lwrite(EngineDev E, int only) {
    const int g = blockIdx.x * kTilesPerBlock + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= E.ntiles) return;
    const int s = E.tile_sys[g];
    if (s < 0 || (only >= 0 && s != only)) return;
    const SysConst& S = E.sys[s];
    SysState* st = S.st;
    const int I = g - S.tile_base;
    if (I >= S.T) return;
    const ListTest T = make_test(S, 1, (float)st->L);
    const float4 oI = *reinterpret_cast<const float4*>(&S.torgf[4 * I]);
    const float hI[3] = {S.thalf[3 * I], S.thalf[3 * I + 1], S.thalf[3 * I + 2]};
    int* lst = S.cl->list;
    int out = S.cl->start[I];
    cluster_tiles(S, I, lane, T, oI, hI, [&](int e) {
        const unsigned m = __ballot_sync(0xffffffffu, e >= 0);
        if (e >= 0) lst[out + __popc(m & ((1u << lane) - 1u))] = e;
        out += __popc(m);
    });
}

// ---------------------------------------------------------------- launchers
void launch_decide(const EngineHost& H, cudaStream_t s, int forced_only, int only,
                   cudaGraphConditionalHandle cond_cell, cudaGraphConditionalHandle cond_list, bool set_cond,
                   cudaGraphConditionalHandle cond_var, bool set_var) {
    H.rec("decide", s);
    launch_dep(k_decide, 1, 1024, s, H.dev, forced_only, only, cond_cell, cond_list, set_cond ? 1 : 0, cond_var,
               set_var ? 1 : 0);
    H.count(1);
}

// Spatial sort and tiles (the cell build).  rec: per-kernel timing events
// (not inside conditional graph nodes, which hold kernels only).
void launch_cell_build(const EngineHost& H, cudaStream_t s, bool rec) {
    const EngineDev& E = H.dev;
    const int nb = (E.ntiles + kTilesPerBlock - 1) / kTilesPerBlock;
    const int nscan = (int)((E.nbins_total + kScanChunk - 1) / kScanChunk);
    if (rec) H.rec("hist", s);
    launch_dep(k_hist, nb, kBlock, s, E);
    if (rec) H.rec("scan", s);
    launch_dep(k_scan_reduce, nscan, 1024, s, E);
    launch_dep(k_scan_bins, nscan, 1024, s, E);
    if (rec) H.rec("scatter", s);
    launch_dep(k_scatter, nb, kBlock, s, E);
    if (rec) H.rec("move", s);
    launch_dep(k_move, nb, kBlock, s, E);
    if (rec) H.rec("tiles", s);
    launch_dep(k_tiles, nb, kBlock, s, E);
    H.count(6);
}

// Super-tile boxes and tile-pair lists (+ per-particle Verlet lists).
void launch_list_build(const EngineHost& H, cudaStream_t s, bool rec) {
    const EngineDev& E = H.dev;
    const int nb = (E.ntiles + kTilesPerBlock - 1) / kTilesPerBlock;
    if (rec) H.rec("lists", s);
    launch_dep(k_super, nb, kBlock, s, E);
    launch_dep(k_lbuild, nb, kBlock, s, E, H.precision == 0 ? 1 : 0);
    H.count(2);
    if (H.any_verlet) {
        if (rec) H.rec("verlet_lists", s);
        launch_dep(k_vbuild, E.ntiles, kVB * 32, s, E);
        H.count(1);
    }
}

// Decision and rebuild launched directly (outside a step graph): the rebuild
// kernels run and return at once unless a system rebuilds.
void launch_rebuild(const EngineHost& H, cudaStream_t s, int forced_only, int only) {
    launch_decide(H, s, forced_only, only, 0, 0, false, 0, false);
    launch_cell_build(H, s, true);
    launch_list_build(H, s, true);
}

// phase 0: count and scan (host then checks capacity); phase 1: write.
void launch_cluster_lists(const EngineHost& H, cudaStream_t s, int phase, int only) {
    const EngineDev& E = H.dev;
    const int nb = (E.ntiles + kTilesPerBlock - 1) / kTilesPerBlock;
    if (phase == 0) {
        H.rec("cl_lcount", s);
        k_lcount<<<nb, kBlock, 0, s>>>(E, only);
        k_lscan<<<E.nsys, 1024, 0, s>>>(E, only);
        H.count(2);
    } else {
        H.rec("cl_lwrite", s);
        k_lwrite<<<nb, kBlock, 0, s>>>(E, only);
        H.count(1);
    }
}

}  // namespace pasta
