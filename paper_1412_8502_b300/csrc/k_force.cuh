// Pair forces of Eq. (1) (Sec. II.A): nuclear term for every pair inside
// r_nuc, screened Coulomb for proton pairs inside r_C, nearest periodic
// image.
//
// Split precision: every pair is evaluated once and its force applied to
// both particles (Newton's third law; the paper's GPU kernel instead sums
// every target over all its sources, Sec. II.B.1).  Work unit: one warp per
// work item, a part of a 32-particle target tile I's half tile-pair list
// (each unordered tile pair is listed once): a proton tile gives four items
// (two halves of its near entries, and two of its Coulomb-only entries), a
// neutron tile one, or two halves of its list in dilute systems; the four
// warps of a block take the same part of four adjacent tiles.  A tile's
// first item first evaluates the tile with itself (broadcast sources, no
// reaction).  For each listed source
// tile J every lane loads one source (cp.async, two entries in flight), moves
// it to the periodic image next to I, and tests it against two boxes around
// the current positions of I's targets 0-15 and 16-31 with the bare cutoffs.
// Sources that pass are compacted (ballot + popc) into shared-memory queues,
// one per pair class: proton-proton with the nuclear term (PPN), proton-
// proton Coulomb only (PPC), unlike species (nuclear, b - c) and like species
// (nuclear, b + c).  A queue holding 32 sources is evaluated as a rotated
// block: lanes l and l ^ 16 hold the same two targets (j = l mod 16 and
// j + 16), the half-warps take 16 sources each, and at step k lane l pairs
// both targets with source (l + k) mod 16 of its half and passes the running
// reaction on that source one lane on with a shuffle; after 16 steps each
// lane holds the whole reaction on one source.  Target sums are plain FP32
// sums of the block partials (energies Kahan-compensated).  All force
// contributions go to per-particle 64-bit fixed-point accumulators
// (2^-32 MeV/fm) with integer atomics, so the result does not depend on their
// order; the closing kick (or k_force_fix) turns them into FP32 forces and
// clears them.
//
// Precision: positions are FP32 pairs hi + lo of the image nearest the tile
// origin (hi rounded to 24 bits, lo the rounded remainder: 48 significant
// bits); periodic shifts of sources use an error-free two-sum, so a
// separation dx = (hi_i - hi_j) + (lo_i - lo_j) carries FP32 rounding of
// order 2^-24 |dx|, whatever the box size.  Pair arithmetic is FP32; far
// Coulomb-only pairs (beyond r_nuc + skin/2 of the target box) use the hi
// part only, an error below 1e-4 fm at r > 12 fm.  Energies are combined in
// FP64.
//
// FP64 validation mode: full lists, one FP64 lane per target and list
// entry stride, no sharing; an FP32 screen passes the pairs near a cutoff.
//
// Single-exponential nuclear term: with g = exp(-r^2/(2 Lambda)),
// exp(-r^2/Lambda) = g^2, so one ex2 serves both Gaussians of Eq. (1).
#include "kernels.h"

namespace pasta {

namespace {

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

enum PairClass { kPPNuc = 0, kPPCoul = 1, kNucCross = 2, kNucSame = 3 };

// Code variants of the split force pass, chosen per system and step: long
// unrolled loops (kULong: rotated blocks 4 steps, the tile with itself 8
// sources), compact (2 and 2) and minimal (1 and 2), the last also in blocks
// of one warp (k_force_split1: a warp whose item ends frees its slot without
// waiting for the other warps of a block).  Where the far
// Coulomb field dominates (dense states), one block kind runs on most warps
// and the long loops issue best; where nuclear pairs are a large part of the
// work (clustered, dilute states), warps of one SM run several block kinds
// at a time and the long code no longer fits the instruction cache (ncu:
// 6 "no instruction" stalls per issue at rho = 0.00125 against 0.3 in the
// dense state); the smaller variants trade instruction-level parallelism
// for footprint.  All variants do the same arithmetic in the same order.
#ifndef PASTA_N3_UNROLL
#define PASTA_N3_UNROLL 4            // steps unrolled in a rotated block, long variant
#endif
constexpr int kULong = PASTA_N3_UNROLL;
constexpr int kUCompact = 2;
constexpr int kUMinimal = 1;
__host__ __device__ constexpr int self_unroll(int kU) { return kU == kULong ? 8 : 2; }

struct PairConsts {
    float rn2, rc2;          // squared cutoffs
    float kq;                // -1/(2 Lambda ln 2): g = 2^(r2 kq)
    float A2;                // 2a/Lambda
    float a;                 // a
    float Ssame, Scross;     // (b+c)/Lambda, (b-c)/Lambda
    float bsame, bcross;     // b+c, b-c
    float kc;                // -1/(lambda ln 2)
    float l2a;               // log2(alpha)
    float il;                // 1/lambda
    float Lhi, Llo, iLf;     // box side as an exact FP32 pair, 1/L
};

struct Acc {
    float fx, fy, fz;
    float en, ec, w;
    float nn, nc;            // in-range pairs (energy pass only), exact below 2^24
};

struct Kahan {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// One queued source against this lane's target.  kLo: use the low parts.
// In-range contributions are added under predicates (no selects).
template <int kClass, bool kLo, bool kWrap, bool kEnergy>
__device__ __forceinline__ void one_pair(const float4& q, const float4& u, const float4& hi, const float4& lo,
                                         const PairConsts& C, float S, float bS, Acc& acc) {
    constexpr bool self_possible = (kClass == kPPNuc) || (kClass == kNucSame);
    float dx = hi.x - q.x, dy = hi.y - q.y, dz = hi.z - q.z;
    if (kLo) {
        dx += lo.x - u.x;
        dy += lo.y - u.y;
        dz += lo.z - u.z;
    }
    if (kWrap) {
        const float kx = rintf(dx * C.iLf), ky = rintf(dy * C.iLf), kz = rintf(dz * C.iLf);
        dx = fmaf(-C.Llo, kx, fmaf(-C.Lhi, kx, dx));
        dy = fmaf(-C.Llo, ky, fmaf(-C.Lhi, ky, dy));
        dz = fmaf(-C.Llo, kz, fmaf(-C.Lhi, kz, dz));
    }
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    // in-range masks as 0/1 factors: branch-free predication of the updates
    float fr = 0.0f;
    if (kClass == kPPNuc || kClass == kPPCoul) {
        const float ri = rsqrt_approx(r2);
        const float r = r2 * ri;
        const float ea = ex2_approx(fmaf(r, C.kc, C.l2a));     // alpha e^{-r/lambda}
        const float vc = ea * ri;                             // screened Coulomb V
        const float fc = vc * ri * (ri + C.il);
        bool in = r2 < C.rc2;
        if (self_possible) {
            // the target itself (r2 = 0) gives inf: select, never multiply
            in = in && (r2 > 0.0f);
            fr = in ? fc : 0.0f;
            if (kEnergy) acc.ec += in ? vc : 0.0f;
        } else {
            const float m = in ? 1.0f : 0.0f;
            fr = fc * m;
            if (kEnergy) acc.ec = fmaf(vc, m, acc.ec);
        }
        if (kEnergy) acc.nc += in ? 1.0f : 0.0f;
    }
    if (kClass != kPPCoul) {
        const float gq = ex2_approx(r2 * C.kq);
        bool in = r2 < C.rn2;
        if (self_possible) in = in && (r2 > 0.0f);
        const float gm = in ? gq : 0.0f;
        fr = fmaf(gm, fmaf(C.A2, gq, S), fr);
        if (kEnergy) {
            acc.en = fmaf(gm, fmaf(C.a, gq, bS), acc.en);
            acc.nn += in ? 1.0f : 0.0f;
        }
    }
    acc.fx = fmaf(fr, dx, acc.fx);
    acc.fy = fmaf(fr, dy, acc.fy);
    acc.fz = fmaf(fr, dz, acc.fz);
    if (kEnergy) acc.w = fmaf(fr, r2, acc.w);
}

// The tile against itself: all lanes take source k in turn (broadcast), for
// all 32 sources (compile-time trip count) or the first n (ragged tiles).
template <int kClass, bool kLo, bool kWrap, bool kEnergy, int kU>
__device__ __forceinline__ void pair_block(const float4* __restrict__ qh, const float4* __restrict__ ql, int n,
                                           const float4& hi, const float4& lo, const PairConsts& C, Acc& acc) {
    const float S = (kClass == kNucCross) ? C.Scross : C.Ssame;
    const float bS = (kClass == kNucCross) ? C.bcross : C.bsame;
    if (n == kTile) {
#pragma unroll self_unroll(kU)
        for (int k = 0; k < kTile; ++k)
            one_pair<kClass, kLo, kWrap, kEnergy>(qh[k], kLo ? ql[k] : qh[k], hi, lo, C, S, bS, acc);
    } else {
        for (int k = 0; k < n; ++k)
            one_pair<kClass, kLo, kWrap, kEnergy>(qh[k], kLo ? ql[k] : qh[k], hi, lo, C, S, bS, acc);
    }
}

// error-free a + b = s + e
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

constexpr int kForceWarps = 4;   // warps (work items) per block
static_assert(kForceWarps == kItemGroup, "a block takes one item of each tile of a group");
// Resident blocks per SM asked of the register allocator: 5 for the passes
// without energies (96 registers, 12-24 bytes of spills; 409,600 dense
// start: long 2.127 -> 2.088 ms, compact 2.237 -> 2.104, minimal 2.274 ->
// 2.137; step 4,000: compact and minimal 8% faster, long 0.7% slower), 4 for
// the energy passes (at 5 their spills and the smaller L1 beside the queues
// made them 1-14% slower).
#ifndef PASTA_FORCE_MIN_BLOCKS
#define PASTA_FORCE_MIN_BLOCKS 4
#endif
#ifndef PASTA_FORCE_MIN_BLOCKS_NOENERGY
#define PASTA_FORCE_MIN_BLOCKS_NOENERGY 5
#endif
constexpr int kQ = 2 * kTile;    // queue capacity
#ifndef PASTA_FORCE_STAGES
#define PASTA_FORCE_STAGES 2
#endif
constexpr int kStages = PASTA_FORCE_STAGES;   // source tiles in flight per warp (cp.async)
constexpr float kUnfixF = 1.0f / 4294967296.0f;   // force accumulators count 2^-32 MeV/fm
constexpr float kForceMax = 1.0e9f;          // |partial force| beyond this (MeV/fm) is an error

struct WarpQueues {
    float4 h[3][kQ];             // 0: PPN / like species, 1: PPC, 2: unlike species
    float4 l[2][kQ];             // low parts of queues 0 and 2 (PPC uses the high parts only)
    float4 dh[2 * kTile];        // block being evaluated, stored twice (rotated reads)
    float4 dl[2 * kTile];
    float4 sh[kStages][kTile];   // staged source tiles (high parts)
    float4 sl[kStages][kTile];   // staged source tiles (low parts)
    int sJ[kStages];             // staged tile index | shift code << 24 | nuclear flag
    float4 box[4];               // half-tile boxes of the targets: centre A, half A, centre B, half B
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int kN>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(kN) : "memory"); }

// A lane's sums over the blocks of a work item.  The forces are plain FP32
// sums of block partials: a block partial carries the rounding of its 32
// pair terms, and adding a few hundred partials (each a small fraction of the
// total in the far Coulomb field) adds a relative error of order 1e-7 of the
// largest partial, far below the 1e-5 force tolerance.  Energies, summed
// over the whole system, are Kahan-compensated.
struct Totals {
    float f0x = 0.f, f0y = 0.f, f0z = 0.f;   // this lane's share of the force on target j = lane mod 16
    float f1x = 0.f, f1y = 0.f, f1z = 0.f;   // ... and on target j + 16
    Kahan ken, kec, kw;
    int nn = 0, nc = 0;          // unique in-range pairs of the rotated blocks
    int nn2 = 0, nc2 = 0;        // ordered in-range pairs of the tile with itself
    int cand = 0;                // unique candidate pairs
    bool bad = false;            // a reaction partial was not finite or out of range
};

struct EAcc {
    float en, ec, w;
    float nn, nc;                // in-range pairs (energy pass only), exact below 2^24
};

// f in units of 2^-32 MeV/fm, rounded to nearest (|f| < 2^31; larger values
// are flagged as errors by the callers).  The hardware conversion issues at
// the FP64 rate but takes one issue slot; an integer construction from the
// bits of f took about fifteen and made the force pass 19% slower.
__device__ __forceinline__ long long to_fix(float f) { return __float2ll_rn(f * 4294967296.0f); }

// Warp total of one FP32 value per lane, compensated (two-sum tree), as FP64.
__device__ __forceinline__ double warp_sum_f(float v) {
    float s = v, c = 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float so = __shfl_xor_sync(0xffffffffu, s, o), co = __shfl_xor_sync(0xffffffffu, c, o);
        float t, e;
        two_sum(s, so, t, e);
        s = t;
        c = c + co + e;
    }
    return (double)s + (double)c;
}

__device__ __forceinline__ void red_add(long long* a, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(a), (unsigned long long)v);
}

// One pair of a rotated block: returns the scalar fr with F_target += fr d
// and F_source -= fr d, where d = x_target - x_source; adds fr d to the
// target sums (fx, fy, fz) and the energies to e.  kSel: masks by select
// (partial blocks, whose unused slots hold zeros); otherwise by multiplying
// with 0/1 (every slot is a real source, never the target).
template <int kClass, bool kLo, bool kWrap, bool kEnergy, bool kSel>
__device__ __forceinline__ float pair_n3(const float4& q, const float4& u, const float4& hi, const float4& lo,
                                         const PairConsts& C, float S, float bS, bool ok, float& fx, float& fy,
                                         float& fz, EAcc& e, float& dx, float& dy, float& dz) {
    dx = hi.x - q.x;
    dy = hi.y - q.y;
    dz = hi.z - q.z;
    if (kLo) {
        dx += lo.x - u.x;
        dy += lo.y - u.y;
        dz += lo.z - u.z;
    }
    if (kWrap) {
        const float kx = rintf(dx * C.iLf), ky = rintf(dy * C.iLf), kz = rintf(dz * C.iLf);
        dx = fmaf(-C.Llo, kx, fmaf(-C.Lhi, kx, dx));
        dy = fmaf(-C.Llo, ky, fmaf(-C.Lhi, ky, dy));
        dz = fmaf(-C.Llo, kz, fmaf(-C.Lhi, kz, dz));
    }
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    float fr = 0.0f;
    if (kClass == kPPNuc || kClass == kPPCoul) {
        const float ri = rsqrt_approx(r2);
        const float r = r2 * ri;
        const bool in = ok && r2 < C.rc2;
        if (kSel) {
            const float ea = ex2_approx(fmaf(r, C.kc, C.l2a));     // alpha e^{-r/lambda}
            const float vc = ea * ri;                             // screened Coulomb V
            const float fc = vc * ri * (ri + C.il);
            fr = in ? fc : 0.0f;
            if (kEnergy) e.ec += in ? vc : 0.0f;
        } else {
            // out of range: 2^-inf = +0 exactly, so V and the force vanish
            // (ri is finite: a real source is never on the target)
            const float arg = in ? fmaf(r, C.kc, C.l2a) : -INFINITY;
            const float ea = ex2_approx(arg);
            const float vc = ea * ri;
            fr = vc * ri * (ri + C.il);
            if (kEnergy) e.ec += vc;
        }
        if (kEnergy && in) e.nc += 1.0f;
    }
    if (kClass != kPPCoul) {
        const float gq = ex2_approx(r2 * C.kq);
        const bool in = ok && r2 < C.rn2;
        const float gm = in ? gq : 0.0f;
        fr = fmaf(gm, fmaf(C.A2, gq, S), fr);
        if (kEnergy) e.en = fmaf(gm, fmaf(C.a, gq, bS), e.en);
        if (kEnergy && in) e.nn += 1.0f;
    }
    fx = fmaf(fr, dx, fx);
    fy = fmaf(fr, dy, fy);
    fz = fmaf(fr, dz, fz);
    if (kEnergy) e.w = fmaf(fr, r2, e.w);
    return fr;
}

// The warp's targets for the rotated blocks: lanes l and l ^ 16 both hold
// targets j = l mod 16 and j + 16 (empty lanes of a ragged tile sit on a real
// particle and are masked off by t0ok / t1ok).
struct Targets {
    float4 h0, l0, h1, l1;
    bool ok0, ok1;
};

// A block of n <= 32 queued sources against the warp's 32 targets, every pair
// once.  Half-warp h = l >> 4 takes sources 16h .. 16h + 15 (stored in Q.dh /
// Q.dl as dh[32h + i] = source 16h + i mod 16, so rotated reads need no
// index arithmetic).  At step k lane l pairs both of its targets with source
// 16h + (j + k) mod 16 and adds the two reactions to registers that rotate
// one lane down within the half after every step: after 16 steps lane l holds
// the whole reaction on source 16h + j.  One source load and one rotation
// serve two pairs.
// cross: unlike species (b - c), chosen at run time so that like and unlike
// nuclear blocks share one instance of the code.
template <int kClass, bool kLo, bool kWrap, bool kEnergy, bool kFull, int kU>
__device__ __forceinline__ void n3_block(const WarpQueues& Q, int n, int lane, const Targets& X,
                                         const PairConsts& C, Totals& T, long long* facc, int N, bool cross) {
    const float S = cross ? C.Scross : C.Ssame;
    const float bS = cross ? C.bcross : C.bsame;
    float f0x = 0.f, f0y = 0.f, f0z = 0.f, f1x = 0.f, f1y = 0.f, f1z = 0.f;
    EAcc e{0.f, 0.f, 0.f, 0.f, 0.f};
    float rx = 0.0f, ry = 0.0f, rz = 0.0f;
    const int half = lane & 16, j = lane & 15;
    const float4* ph = Q.dh + 2 * half + j;
    const float4* pl = Q.dl + 2 * half + j;
    const int from = half | ((lane + 1) & 15);
    auto step = [&](int k) {
        const float4 q = ph[k];
        const float4 u = kLo ? pl[k] : q;
        const bool sv = kFull || ((half | ((j + k) & 15)) < n);
        float dx, dy, dz;
        const float fr0 = pair_n3<kClass, kLo, kWrap, kEnergy, !kFull>(q, u, X.h0, X.l0, C, S, bS, X.ok0 && sv, f0x,
                                                                         f0y, f0z, e, dx, dy, dz);
        rx = fmaf(-fr0, dx, rx);
        ry = fmaf(-fr0, dy, ry);
        rz = fmaf(-fr0, dz, rz);
        const float fr1 = pair_n3<kClass, kLo, kWrap, kEnergy, !kFull>(q, u, X.h1, X.l1, C, S, bS, X.ok1 && sv, f1x,
                                                                         f1y, f1z, e, dx, dy, dz);
        rx = __shfl_sync(0xffffffffu, fmaf(-fr1, dx, rx), from);
        ry = __shfl_sync(0xffffffffu, fmaf(-fr1, dy, ry), from);
        rz = __shfl_sync(0xffffffffu, fmaf(-fr1, dz, rz), from);
    };
    if (kWrap) {                 // longer bodies: half the unrolling
#pragma unroll (kU + 1) / 2
        for (int k = 0; k < 16; ++k) step(k);
    } else {
#pragma unroll kU
        for (int k = 0; k < 16; ++k) step(k);
    }
    if ((half | j) < n) {
        const int slot = __float_as_int(ph[0].w);
        T.bad |= !(fabsf(rx) < kForceMax && fabsf(ry) < kForceMax && fabsf(rz) < kForceMax);
        red_add(facc + slot, to_fix(rx));
        red_add(facc + N + slot, to_fix(ry));
        red_add(facc + 2 * N + slot, to_fix(rz));
    }
    T.f0x += f0x;
    T.f0y += f0y;
    T.f0z += f0z;
    T.f1x += f1x;
    T.f1y += f1y;
    T.f1z += f1z;
    if (kEnergy) {
        // a class without a term adds nothing to that term's sums
        if (kClass != kPPCoul) T.ken.add(e.en);
        if (kClass == kPPNuc || kClass == kPPCoul) T.kec.add(e.ec);
        T.kw.add(e.w);
        if (kClass != kPPCoul) T.nn += (int)e.nn;
        if (kClass == kPPNuc || kClass == kPPCoul) T.nc += (int)e.nc;
    }
    T.cand += n * kTile;
}

template <int kClass, bool kLo, bool kWrap, bool kEnergy, int kU>
__device__ __forceinline__ void n3_any(const WarpQueues& Q, int n, int lane, const Targets& X, const PairConsts& C,
                                       Totals& T, long long* facc, int N, bool cross = false) {
    // Without per-pair wrapping the unused slots of a partial block hold a
    // far pad position (drain), whose pair terms vanish exactly (2^-huge = +0,
    // out of range): the full-block code serves every block, which keeps the
    // instruction footprint of the pass small.
    if (n == kTile || !kWrap) n3_block<kClass, kLo, kWrap, kEnergy, true, kU>(Q, n, lane, X, C, T, facc, N, cross);
    else n3_block<kClass, kLo, kWrap, kEnergy, false, kU>(Q, n, lane, X, C, T, facc, N, cross);
}

// Evaluate the first min(cnt, 32) entries of queue q, shift the rest down.
template <bool kWrap, bool kEnergy, int kU>
__device__ __forceinline__ void drain(WarpQueues& Q, int q, int cls, int& cnt, int lane, const Targets& X,
                                      const PairConsts& C, Totals& T, long long* facc, int N) {
    __syncwarp();
    const int n = min(cnt, kTile);
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    // unused slots: zeros with per-pair wrapping (the partial-block code masks
    // them), else a pad 1e9 fm away (all terms underflow to zero)
    const float4 pad = kWrap ? zero : make_float4(kPad, kPad, kPad, 0.f);
    const int half = lane & 16, j = lane & 15;
    const float4 h = lane < n ? Q.h[q][lane] : pad;
    Q.dh[2 * half + j] = h;
    Q.dh[2 * half + 16 + j] = h;
    if (q != 1) {
        const float4 l = lane < n ? Q.l[q >> 1][lane] : zero;
        Q.dl[2 * half + j] = l;
        Q.dl[2 * half + 16 + j] = l;
    }
    __syncwarp();
    const int rest = cnt - n;
    if (lane < rest) {
        Q.h[q][lane] = Q.h[q][kTile + lane];
        if (q != 1) Q.l[q >> 1][lane] = Q.l[q >> 1][kTile + lane];
    }
    cnt = rest;
    __syncwarp();
    switch (cls) {
        case kPPNuc: n3_any<kPPNuc, true, kWrap, kEnergy, kU>(Q, n, lane, X, C, T, facc, N); break;
        case kPPCoul: n3_any<kPPCoul, false, kWrap, kEnergy, kU>(Q, n, lane, X, C, T, facc, N); break;
        default: n3_any<kNucSame, true, kWrap, kEnergy, kU>(Q, n, lane, X, C, T, facc, N, cls == kNucCross); break;
    }
}

__device__ __forceinline__ void push(WarpQueues& Q, int q, bool pred, int& cnt, int lane, const float4& h,
                                     const float4& l) {
    const unsigned m = __ballot_sync(0xffffffffu, pred);
    if (pred) {
        const int pos = cnt + __popc(m & ((1u << lane) - 1u));
        Q.h[q][pos] = h;
        if (q != 1) Q.l[q >> 1][pos] = l;
    }
    cnt += __popc(m);
}

// Work item v of a system (see item_index): a part of a proton tile's near
// entries (the first with the tile itself) or of its Coulomb-only entries, or
// a part of a neutron tile's list (the first with the tile itself).
template <bool kWrap, bool kEnergy, int kU>
__device__ __forceinline__ void force_item(const SysConst& S, const PairF& P, int v, WarpQueues& Q) {
    const int lane = threadIdx.x & 31;
    const int Pi = proton_items(S.Tp);
    SysState* st = S.st;
    const double L = st->L;
    int I, c, nparts;              // proton tiles: part c of kPChunks; neutron tiles: part c of nparts
    if (v < Pi) {
        const int b = v / kItemGroup;
        I = (b / kPChunks) * kItemGroup + v % kItemGroup;
        c = b % kPChunks;
        nparts = kPChunks;
        if (I >= S.Tp) return;     // past the last proton tile of the group
    } else {
        // split: the halves of kItemGroup adjacent tiles side by side; whole
        // lists: one item per tile, the unused items at the end of the pass
        const int w = v - Pi;
        if ((double)S.N < kSplitRho * L * L * L) {
            const int b = w / kItemGroup;
            I = S.Tp + (b / kNChunks) * kItemGroup + w % kItemGroup;
            c = b % kNChunks;
            nparts = kNChunks;
        } else {
            I = S.Tp + w;
            c = 0;
            nparts = 1;
        }
        if (I >= S.T) return;
    }
    const int N = S.N;
    long long* facc = S.facc;

    PairConsts C;
    C.rn2 = P.rn2;
    C.rc2 = P.rc2;
    C.kq = P.kq;
    C.A2 = P.A2;
    C.a = P.a;
    C.Ssame = P.Ssame;
    C.Scross = P.Scross;
    C.bsame = P.bsame;
    C.bcross = P.bcross;
    C.kc = P.kc;
    C.l2a = P.l2a;
    C.il = P.il;
    // L as an exact FP32 pair; 1/L only picks images (FP32 division)
    const float Lhi = __double2float_rn(L), Llo = __double2float_rn(L - (double)Lhi);
    C.Lhi = Lhi;
    C.Llo = Llo;
    C.iLf = 1.0f / Lhi;
    // source filter radii around I's box: cutoff + skin/2 (+ FP32 margin)
    const float Rn2 = P.Rn2, Rc2 = P.Rc2;

    const int p = tile_slot0(S, I) + lane;
    const int nv = tile_end(S, I) - tile_slot0(S, I);
    const bool valid = lane < nv;
    const int j = lane & 15;
    // Empty lanes of a ragged tile sit on particle 0 of the tile (a finite,
    // in-box position, never a source) and their pairs are masked off, so
    // they add no reaction to real sources.
    Targets X;
    {
        const float4 a0 = S.xhi[I * kTile], b0 = S.xlo[I * kTile];
        X.ok0 = j < nv;
        X.ok1 = j + 16 < nv;
        X.h0 = X.ok0 ? S.xhi[I * kTile + j] : a0;
        X.l0 = X.ok0 ? S.xlo[I * kTile + j] : b0;
        X.h1 = X.ok1 ? S.xhi[I * kTile + j + 16] : a0;
        X.l1 = X.ok1 ? S.xlo[I * kTile + j + 16] : b0;
    }
    // Boxes of the targets' current positions, one per half tile (targets
    // j = 0..15 in .x of the lanes' pairs, j + 16 in .y; a lane on an empty
    // slot sits on a real particle of the tile), widened by 1e-3 fm for the
    // low parts and FP32 rounding.  A source is kept when it is within the
    // bare cutoff of either box: the union of the two regions is smaller than
    // the region around the tile's single box wherever the tile is not
    // box-shaped, and the rebuild-time box would need the skin on top.
    // (kept in shared memory: registers are the scarce resource here)
    {
        const float a0[3] = {X.h0.x, X.h0.y, X.h0.z}, a1[3] = {X.h1.x, X.h1.y, X.h1.z};
        float cA[3], hA[3], cB[3], hB[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float la = fkey_inv(__reduce_min_sync(0xffffffffu, fkey(a0[a])));
            const float ua = fkey_inv(__reduce_max_sync(0xffffffffu, fkey(a0[a])));
            const float lb = fkey_inv(__reduce_min_sync(0xffffffffu, fkey(a1[a])));
            const float ub = fkey_inv(__reduce_max_sync(0xffffffffu, fkey(a1[a])));
            cA[a] = 0.5f * (la + ua);
            hA[a] = 0.5f * (ua - la) + 1e-3f;
            cB[a] = 0.5f * (lb + ub);
            hB[a] = 0.5f * (ub - lb) + 1e-3f;
        }
        if (lane == 0) {
            Q.box[0] = make_float4(cA[0], cA[1], cA[2], 0.0f);
            Q.box[1] = make_float4(hA[0], hA[1], hA[2], 0.0f);
            Q.box[2] = make_float4(cB[0], cB[1], cB[2], 0.0f);
            Q.box[3] = make_float4(hB[0], hB[1], hB[2], 0.0f);
        }
        __syncwarp();
    }
    // The system's constants the entry loop needs, read once: the loop's
    // stores and atomics would otherwise have them loaded again for every
    // entry (3% of the dense pass).
    const int Tp = S.Tp, Tl = S.T;
    const bool Ip = I < Tp;
    const bool ppc = Ip && S.coulomb == 1;     // proton tile, Coulomb term on the lists
    const int cls0 = ppc ? kPPNuc : kNucSame;
    const float4* const xhi_g = S.xhi;
    const float4* const xlo_g = S.xlo;
    const int* lst = S.list + (long long)I * S.T;
    const int nl = S.lcount[I], nn = S.lnear[I];
    int e0, e1;
    if (!Ip) {
        static_assert(kNChunks == 2, "neutron tiles: the whole list or its two halves");
        e0 = (nparts == 1 || c == 0) ? 0 : nl / 2;
        e1 = (nparts == 2 && c == 0) ? nl / 2 : nl;
    } else if (c < kPNear) {
        e0 = (int)((long long)nn * c / kPNear);
        e1 = (int)((long long)nn * (c + 1) / kPNear);
    } else {
        const int nf = nl - nn;
        e0 = nn + (int)((long long)nf * (c - kPNear) / (kPChunks - kPNear));
        e1 = nn + (int)((long long)nf * (c - kPNear + 1) / (kPChunks - kPNear));
    }

    Totals T;
    int c0 = 0, c1 = 0, c2 = 0;

    // Stage entry e: tile index, periodic shift toward I and nuclear flag
    // (lane 0 stores them), then this lane's source coordinates (cp.async;
    // the low parts only when the nuclear term is reachable).
    auto stage = [&](int e) {
        const int slot = (int)((unsigned)(e - e0) % kStages);
        const int ent = lst[e < nn ? e : Tl - 1 - (e - nn)];
        const int J = ent & kJMask;
        if (lane == 0) Q.sJ[slot] = ent;
        cp_async16(&Q.sh[slot][lane], &xhi_g[J * kTile + lane]);
        if ((ent & kNucBit) || !(ppc && J < Tp)) cp_async16(&Q.sl[slot][lane], &xlo_g[J * kTile + lane]);
    };
    for (int d = 0; d < kStages - 1; ++d) {
        if (e0 + d < e1) stage(e0 + d);
        cp_async_commit();
    }

    // The tile with itself (the lists leave it out): lane l takes target l
    // against every particle of the tile, so no reaction is added and the
    // energies count each pair twice.
    float sfx = 0.0f, sfy = 0.0f, sfz = 0.0f;
    if (c == 0) {
        const float4 hs = (lane & 16) ? X.h1 : X.h0, ls = (lane & 16) ? X.l1 : X.l0;
        Q.dh[lane] = hs;
        Q.dl[lane] = ls;
        __syncwarp();
        Acc a{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (cls0 == kPPNuc) pair_block<kPPNuc, true, kWrap, kEnergy, kU>(Q.dh, Q.dl, nv, hs, ls, C, a);
        else pair_block<kNucSame, true, kWrap, kEnergy, kU>(Q.dh, Q.dl, nv, hs, ls, C, a);
        sfx = a.fx;
        sfy = a.fy;
        sfz = a.fz;
        if (kEnergy) {
            T.ken.add(valid ? 0.5f * a.en : 0.0f);
            T.kec.add(valid ? 0.5f * a.ec : 0.0f);
            T.kw.add(valid ? 0.5f * a.w : 0.0f);
            T.nn2 += (int)a.nn;
            T.nc2 += (int)a.nc;
        }
        T.cand += nv * (nv - 1) / 2;
    }

    for (int e = e0; e < e1; ++e) {
        if (e + kStages - 1 < e1) stage(e + kStages - 1);
        cp_async_commit();
        cp_async_wait<kStages - 1>();
        __syncwarp();
        const int slot = (int)((unsigned)(e - e0) % kStages);
        const int tag = Q.sJ[slot];
        const int Jk = tag & kJMask;
        const int shk = (tag >> kShiftPos) & 63;
        const bool nucflag = (tag & kNucBit) != 0;
        float4 h = Q.sh[slot][lane];
        const bool Jp = Jk < Tp;
        const bool farc = ppc && Jp && !nucflag;   // Coulomb-only entry
        float4 l = farc ? make_float4(0.f, 0.f, 0.f, 0.f) : Q.sl[slot][lane];
        __syncwarp();
        const bool src_ok = h.x != kPad;
        if (shk != kShiftNone) apply_shift(shk, Lhi, Llo, h, l);
        // squared distance of the source to the nearer half-tile box (small
        // boxes: nearest image)
        float d2h[2];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const float4 cc4 = Q.box[2 * b], hh4 = Q.box[2 * b + 1];
            const float cc[3] = {cc4.x, cc4.y, cc4.z}, hh[3] = {hh4.x, hh4.y, hh4.z};
            float ux = h.x - cc[0], uy = h.y - cc[1], uz = h.z - cc[2];
            if (kWrap) {
                ux = fmaf(-Lhi, rintf(ux * C.iLf), ux);
                uy = fmaf(-Lhi, rintf(uy * C.iLf), uy);
                uz = fmaf(-Lhi, rintf(uz * C.iLf), uz);
            }
            const float gx = fmaxf(fabsf(ux) - hh[0], 0.0f);
            const float gy = fmaxf(fabsf(uy) - hh[1], 0.0f);
            const float gz = fmaxf(fabsf(uz) - hh[2], 0.0f);
            d2h[b] = fmaf(gz, gz, fmaf(gy, gy, gx * gx));
        }
        const float d2 = fminf(d2h[0], d2h[1]);
        if (farc) {                // Coulomb-only entry: every source goes to PPC or nowhere
            push(Q, 1, src_ok && d2 < Rc2, c1, lane, h, l);
            if (c1 >= kTile) drain<kWrap, kEnergy, kU>(Q, 1, kPPCoul, c1, lane, X, C, T, facc, N);
        } else if (ppc && Jp) {
            const bool nuc = src_ok && d2 < Rn2;
            push(Q, 0, nuc, c0, lane, h, l);
            push(Q, 1, src_ok && !nuc && d2 < Rc2, c1, lane, h, l);
            if (c0 >= kTile) drain<kWrap, kEnergy, kU>(Q, 0, kPPNuc, c0, lane, X, C, T, facc, N);
            if (c1 >= kTile) drain<kWrap, kEnergy, kU>(Q, 1, kPPCoul, c1, lane, X, C, T, facc, N);
        } else if (Ip != Jp) {
            push(Q, 2, src_ok && d2 < Rn2, c2, lane, h, l);
            if (c2 >= kTile) drain<kWrap, kEnergy, kU>(Q, 2, kNucCross, c2, lane, X, C, T, facc, N);
        } else {
            push(Q, 0, src_ok && d2 < Rn2, c0, lane, h, l);
            if (c0 >= kTile) drain<kWrap, kEnergy, kU>(Q, 0, cls0, c0, lane, X, C, T, facc, N);
        }
    }
    cp_async_wait<0>();
    // flush the partial queues (< 32 entries each)
    if (c0 > 0) drain<kWrap, kEnergy, kU>(Q, 0, cls0, c0, lane, X, C, T, facc, N);
    if (c1 > 0) drain<kWrap, kEnergy, kU>(Q, 1, kPPCoul, c1, lane, X, C, T, facc, N);
    if (c2 > 0) drain<kWrap, kEnergy, kU>(Q, 2, kNucCross, c2, lane, X, C, T, facc, N);

    // Target l = j + 16 (l >> 4): this lane's share plus its partner's
    // (lane l ^ 16 holds the same two targets), plus the tile's own pairs.
    const bool upper = (lane & 16) != 0;
    const float m0x = T.f0x, m0y = T.f0y, m0z = T.f0z;
    const float m1x = T.f1x, m1y = T.f1y, m1z = T.f1z;
    const float ox = __shfl_xor_sync(0xffffffffu, upper ? m0x : m1x, 16);
    const float oy = __shfl_xor_sync(0xffffffffu, upper ? m0y : m1y, 16);
    const float oz = __shfl_xor_sync(0xffffffffu, upper ? m0z : m1z, 16);
    const float fx = ((upper ? m1x : m0x) + ox) + sfx;
    const float fy = ((upper ? m1y : m0y) + oy) + sfy;
    const float fz = ((upper ? m1z : m0z) + oz) + sfz;
    bool bad = T.bad;
    if (valid) {
        bad |= !(fabsf(fx) < kForceMax && fabsf(fy) < kForceMax && fabsf(fz) < kForceMax);
        red_add(facc + p, to_fix(fx));
        red_add(facc + N + p, to_fix(fy));
        red_add(facc + 2 * N + p, to_fix(fz));
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&st->error, 1);
    if (kEnergy) {
        // energies and counts of the rotated blocks were summed over every
        // lane's pairs, empty targets masked; those of the tile's own pairs
        // only over valid lanes
        const double en = warp_sum_f(T.ken.s - T.ken.c);
        const double ec = warp_sum_f(T.kec.s - T.kec.c);
        const double wv = warp_sum_f(T.kw.s - T.kw.c);
        const int cn = __reduce_add_sync(0xffffffffu, 2 * T.nn + (valid ? T.nn2 : 0));   // twice the pairs
        const int cc = __reduce_add_sync(0xffffffffu, 2 * T.nc + (valid ? T.nc2 : 0));
        if (lane == 0) add_energy(st, en, ec, wv, cn, cc, 2ll * T.cand);
    }
}

// kVar: the code variant (0 long, 1 compact, 2 minimal), each its own
// kernel so that the variants do not share one register allocation and code
// layout (one kernel holding all three made the long variant 1.8% slower).
// gate: the launch returns at once unless kVar is this step's selection
// (plain graphs launch all of them).  Block 0 records the start of the pass
// for the tuner.
// Global work item g of the split force pass, taken by one warp (queues Q).
template <bool kEnergy, int kVar>
__device__ __forceinline__ void force_split_item(const EngineDev& E, int only, int g, WarpQueues& Q) {
    constexpr int kU = kVar == 0 ? kULong : kVar == 1 ? kUCompact : kUMinimal;
    constexpr int kUWrap = kVar == 0 ? kULong : kUCompact;                  // per-pair wrap halves it
    if (g >= E.nitems) return;
    const int s = E.item_sys[g];
    if (s < 0 || (only >= 0 && s != only)) return;
    const SysConst& S = E.sys[s];
    if (S.list_kind != 0) return;          // per-particle lists: k_force_verlet
    const int v = g - S.item_base;
    if (v >= S.n_items) return;
    const PairF& P = S.pf;
    if (S.st->need_wrap) force_item<true, kEnergy, kUWrap>(S, P, v, Q);
    else force_item<false, kEnergy, kU>(S, P, v, Q);
}

template <bool kEnergy, int kVar>
__global__ void __launch_bounds__(kForceWarps * 32, kEnergy ? PASTA_FORCE_MIN_BLOCKS : PASTA_FORCE_MIN_BLOCKS_NOENERGY)
    k_force_split(EngineDev E, int only, int gate) {
    __shared__ WarpQueues qs[kForceWarps];
    ForceTune* tu = E.tune;
    if (gate && tu->sel != kVar) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) tu->t_start = global_ns();   // k_force_fix takes the end
    const int g = blockIdx.x * kForceWarps + (threadIdx.x >> 5);
    force_split_item<kEnergy, kVar>(E, only, g, qs[threadIdx.x >> 5]);
}

// The fourth variant: the minimal code, one warp (work item) per block, 16
// blocks per SM with energies, 20 without (96 registers: 0.330 -> 0.310 ms
// at step 19,000 of the 409,600 expansion; with energies 20 were 3-7% slower),
// so that no warp waits for the others of a block.
constexpr int kVarOneWarp = 3;
template <bool kEnergy>
__global__ void __launch_bounds__(32, kEnergy ? 16 : 20) k_force_split1(EngineDev E, int only, int gate) {
    __shared__ WarpQueues qs;
    ForceTune* tu = E.tune;
    if (gate && tu->sel != kVarOneWarp) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) tu->t_start = global_ns();
    force_split_item<kEnergy, 2>(E, only, blockIdx.x, qs);
}

// ---------------------------------------------------------------- Verlet
// Split precision over per-particle Verlet lists (list_kind 1): one block of
// kVW warps per tile; lane l of warp w sums its target over entries
// k = w, w + kVW, ... of its list (two entries in flight), and the warps'
// partial sums are added in warp order (deterministic).  Every neighbour is
// listed on both sides, so no reaction is shared.  Sources are gathered by
// tile slot; the entry's periodic shift is applied with an error-free sum
// and the low parts are read for entries inside the nuclear range + skin,
// so separations are exact as in k_force_split (far Coulomb-only pairs use
// the high parts, as there).  The result goes to the fixed-point
// accumulators (plain stores: one writer per particle), which k_force_fix
// turns into FP32 forces.
constexpr int kVW = 4;

struct VAcc {
    float fx, fy, fz, en, ec, w, nn, nc;
};

template <bool kWrap, bool kEnergy>
__device__ __forceinline__ void verlet_pair(const SysConst& S, int ent, const float4& hi, const float4& lo, bool Ip,
                                            bool coul, int pslots, float Lhi, float Llo, float iLf, VAcc& a) {
    const PairF& P = S.pf;
    const int j = ent & kJMask;
    const int shk = (ent >> kShiftPos) & 63;
    const bool near = (ent & kNucBit) != 0;
    float4 h = S.xhi[j];
    float4 l = near ? S.xlo[j] : make_float4(0.f, 0.f, 0.f, 0.f);
    if (shk != kShiftNone) apply_shift(shk, Lhi, Llo, h, l);
    float dx = hi.x - h.x, dy = hi.y - h.y, dz = hi.z - h.z;
    if (near) {                          // far Coulomb-only pairs: high parts only
        dx += lo.x - l.x;
        dy += lo.y - l.y;
        dz += lo.z - l.z;
    }
    if (kWrap) {
        const float qx = rintf(dx * iLf), qy = rintf(dy * iLf), qz = rintf(dz * iLf);
        dx = fmaf(-Llo, qx, fmaf(-Lhi, qx, dx));
        dy = fmaf(-Llo, qy, fmaf(-Lhi, qy, dy));
        dz = fmaf(-Llo, qz, fmaf(-Lhi, qz, dz));
    }
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    const bool jp = j < pslots;
    float fr = 0.0f;
    if (coul && Ip && jp) {
        const float ri = rsqrt_approx(r2);
        const float ea = ex2_approx(fmaf(r2 * ri, P.kc, P.l2a));
        const float vc = ea * ri;
        const bool in = r2 < P.rc2;
        fr = in ? vc * ri * (ri + P.il) : 0.0f;
        if (kEnergy && in) {
            a.ec += vc;
            a.nc += 1.0f;
        }
    }
    if (near) {
        const float gq = ex2_approx(r2 * P.kq);
        const bool in = r2 < P.rn2;
        const bool same = Ip == jp;
        const float gm = in ? gq : 0.0f;
        fr = fmaf(gm, fmaf(P.A2, gq, same ? P.Ssame : P.Scross), fr);
        if (kEnergy && in) {
            a.en = fmaf(gq, fmaf(P.a, gq, same ? P.bsame : P.bcross), a.en);
            a.nn += 1.0f;
        }
    }
    a.fx = fmaf(fr, dx, a.fx);
    a.fy = fmaf(fr, dy, a.fy);
    a.fz = fmaf(fr, dz, a.fz);
    if (kEnergy) a.w = fmaf(fr, r2, a.w);
}

template <bool kWrap, bool kEnergy>
__device__ __forceinline__ void verlet_tile(const SysConst& S, int I, float (*red)[8][kTile]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    SysState* st = S.st;
    const double L = st->L;
    const int N = S.N;
    const float Lhi = __double2float_rn(L), Llo = __double2float_rn(L - (double)Lhi), iLf = 1.0f / Lhi;
    const int p = tile_slot0(S, I) + lane;
    const bool valid = p < tile_end(S, I);
    const float4 hi = S.xhi[I * kTile + lane], lo = S.xlo[I * kTile + lane];
    const bool Ip = I < S.Tp;
    const bool coul = S.coulomb == 1;
    const int cnt = valid ? S.vcount[I * kTile + lane] : 0;
    const int* vl = S.vlist + S.voff[I] + lane;
    const int width = S.vwidth[I];
    const int pslots = S.Tp * kTile;             // tile slots below this are protons
    Kahan kx, ky, kz, ken, kec, kw;
    int nn = 0, nc = 0;
    // blocks of 16 steps of kVW entries, two entries in flight per step
    for (int k0 = w; k0 < width; k0 += 32 * kVW) {
        VAcc a{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const int k1 = min(cnt, k0 + 32 * kVW);
        for (int k = k0; k < k1; k += 2 * kVW) {
            const bool two = k + kVW < k1;
            const int e0 = vl[32ll * k];
            const int e1 = two ? vl[32ll * (k + kVW)] : 0;
            verlet_pair<kWrap, kEnergy>(S, e0, hi, lo, Ip, coul, pslots, Lhi, Llo, iLf, a);
            if (two) verlet_pair<kWrap, kEnergy>(S, e1, hi, lo, Ip, coul, pslots, Lhi, Llo, iLf, a);
        }
        kx.add(a.fx);
        ky.add(a.fy);
        kz.add(a.fz);
        if (kEnergy) {
            ken.add(a.en);
            kec.add(a.ec);
            kw.add(a.w);
            nn += (int)a.nn;
            nc += (int)a.nc;
        }
    }
    // partial sums of the kVW warps, added in warp order by warp 0
    red[w][0][lane] = kx.s - kx.c;
    red[w][1][lane] = ky.s - ky.c;
    red[w][2][lane] = kz.s - kz.c;
    red[w][3][lane] = ken.s - ken.c;
    red[w][4][lane] = kec.s - kec.c;
    red[w][5][lane] = kw.s - kw.c;
    red[w][6][lane] = __int_as_float(nn);
    red[w][7][lane] = __int_as_float(nc);
    __syncthreads();
    if (w != 0) return;
    float fx = 0.f, fy = 0.f, fz = 0.f, en = 0.f, ec = 0.f, wv = 0.f;
    int tn = 0, tc = 0;
    for (int q = 0; q < kVW; ++q) {
        fx += red[q][0][lane];
        fy += red[q][1][lane];
        fz += red[q][2][lane];
        en += red[q][3][lane];
        ec += red[q][4][lane];
        wv += red[q][5][lane];
        tn += __float_as_int(red[q][6][lane]);
        tc += __float_as_int(red[q][7][lane]);
    }
    bool bad = false;
    if (valid) {
        bad = !(fabsf(fx) < kForceMax && fabsf(fy) < kForceMax && fabsf(fz) < kForceMax);
        S.facc[p] = to_fix(fx);
        S.facc[N + p] = to_fix(fy);
        S.facc[2 * N + p] = to_fix(fz);
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&st->error, 1);
    if (kEnergy) {
        // every pair is in both particles' lists: halve the sums
        const double e_n = warp_sum_f(en), e_c = warp_sum_f(ec), w_v = warp_sum_f(wv);
        const int cn = __reduce_add_sync(0xffffffffu, tn), cc = __reduce_add_sync(0xffffffffu, tc);
        const int ca = __reduce_add_sync(0xffffffffu, cnt);
        if (lane == 0) add_energy(st, 0.5 * e_n, 0.5 * e_c, 0.5 * w_v, cn, cc, ca);
    }
}

template <bool kEnergy>
__global__ void __launch_bounds__(kVW * 32) k_force_verlet(EngineDev E, int only) {
    __shared__ float red[kVW][8][kTile];
    const int g = blockIdx.x;
    if (g >= E.ntiles) return;
    const int s = E.tile_sys[g];
    if (s < 0 || (only >= 0 && s != only)) return;
    const SysConst& S = E.sys[s];
    if (S.list_kind != 1) return;
    const int I = g - S.tile_base;
    if (I >= S.T) return;
    if (S.st->need_wrap) verlet_tile<true, kEnergy>(S, I, red);
    else verlet_tile<false, kEnergy>(S, I, red);
}

// Fixed-point accumulators -> FP32 forces (rounded once), and back to zero
// for the next pass.  One warp per tile, one lane per particle.
__global__ void __launch_bounds__(kForceWarps * 32) k_force_fix(EngineDev E, int only, int out_alt) {
    // duration of the force pass that this launch follows (device tuner)
    if (blockIdx.x == 0 && threadIdx.x == 0) E.tune->t_last = global_ns() - E.tune->t_start;
    const int g = blockIdx.x * kForceWarps + (threadIdx.x >> 5);
    if (g >= E.ntiles) return;
    const int s = E.tile_sys[g];
    if (s < 0 || (only >= 0 && s != only)) return;
    const SysConst& S = E.sys[s];
    const int I = g - S.tile_base;
    if (I >= S.T) return;
    const int p = tile_slot0(S, I) + (threadIdx.x & 31);
    if (p >= tile_end(S, I)) return;
    const SysState* st = S.st;
    const int N = S.N;
    // all loads first (the stores below may not be ordered before them)
    long long v[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = S.facc[c * N + p];
    float* F = S.f32[out_alt ? (st->cur ^ 1) : st->cur];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        S.facc[c * N + p] = 0;
        // one rounding of v to FP32 (|v| < 2^53: the same value as rounding
        // v 2^-32 from FP64), then an exact power-of-two scale
        F[c * N + p] = __ll2float_rn(v[c]) * kUnfixF;
    }
}

// ---------------------------------------------------------------- FP64
// Validation mode: FP64 positions, per-pair nearest image, FP64 exp/sqrt,
// full lists (each pair evaluated for both particles, no sharing).  One
// block of kFW warps per target tile: warp w takes list entries w, w + kFW,
// ..., lane l target l of the tile; the warps' partial sums are added in
// warp order (deterministic).  A pair first passes an FP32 screen on the
// tile-frame hi + lo positions against the largest cutoff that applies plus
// a band far wider than the FP32 error of the screen (2e-3 relative +
// 1e-3 fm^2), so only pairs that may lie inside a cutoff reach the FP64
// arithmetic, whose own comparisons decide.
constexpr int kFW = 16;

template <bool kEnergy>
__global__ void __launch_bounds__(kFW * 32) k_force_fp64(EngineDev E, int only, int out_alt, int chunks) {
    __shared__ double sb[kFW][3][kTile];
    __shared__ float4 sh[kFW][kTile], sl[kFW][kTile];
    __shared__ double red[kFW][3][kTile];
    __shared__ double ered[kFW][5];
    __shared__ int last;
    // block -> (tile g, chunk ch): with few tiles, chunks of a tile's entries
    // run in separate blocks (entries ch kFW + w, + chunks kFW, ...) and the
    // last block of a tile adds the chunks' partial forces in chunk order
    const int g = blockIdx.x % E.ntiles, ch = blockIdx.x / E.ntiles;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (g >= E.ntiles) return;
    const int s = E.tile_sys[g];
    if (s < 0 || (only >= 0 && s != only)) return;
    const SysConst& S = E.sys[s];
    const int I = g - S.tile_base;
    if (I >= S.T) return;
    SysState* st = S.st;
    const double L = st->L, hL = 0.5 * L;
    const float Lhi = __double2float_rn(L), Llo = __double2float_rn(L - (double)Lhi), iLf = 1.0f / Lhi;
    const int N = S.N;
    const double* x = S.x[st->cur];
    const int p = tile_slot0(S, I) + lane;
    const bool valid = p < tile_end(S, I);
    const double xi = valid ? x[p] : 0.0, yi = valid ? x[N + p] : 0.0, zi = valid ? x[2 * N + p] : 0.0;
    const float4 hi = S.xhi[I * kTile + lane], lo = S.xlo[I * kTile + lane];
    const bool Ip = I < S.Tp;
    const double rn2 = S.r_nuc * S.r_nuc, rc2 = S.r_C * S.r_C;
    const double A2 = 2.0 * S.a / S.Lambda, i2L = 1.0 / (2.0 * S.Lambda), iLam = 1.0 / S.Lambda;
    const double il = 1.0 / S.lambda_s;
    const float lim_n = (float)rn2 * (1.0f + 2e-3f) + 1e-3f;
    const float lim_c = (float)fmax(rn2, rc2) * (1.0f + 2e-3f) + 1e-3f;
    double fx = 0, fy = 0, fz = 0, en = 0, ec = 0, wv = 0;
    int nn = 0, nc = 0;
    const int* lst = S.list + (long long)I * S.T;
    const int e1 = S.lcount[I], nnear = S.lnear[I];
    for (int e = ch * kFW + w; e < e1; e += chunks * kFW) {
        const int J = lst[list_pos(S, e, nnear)] & kJMask;
        const int q = tile_slot0(S, J) + lane;
        const int nq = tile_end(S, J) - tile_slot0(S, J);
        const bool qv = lane < nq;
        __syncwarp();
        sb[w][0][lane] = qv ? x[q] : 0.0;
        sb[w][1][lane] = qv ? x[N + q] : 0.0;
        sb[w][2][lane] = qv ? x[2 * N + q] : 0.0;
        sh[w][lane] = S.xhi[J * kTile + lane];
        sl[w][lane] = S.xlo[J * kTile + lane];
        __syncwarp();
        const bool Jp = J < S.Tp;
        const bool pp = Ip && Jp && S.coulomb == 1;
        const double bc = (Ip == Jp) ? (S.b + S.c) : (S.b - S.c);
        const float lim = pp ? lim_c : lim_n;
        if (valid) {
            for (int k = 0; k < nq; ++k) {
                if (J == I && k == lane) continue;
                // FP32 screen (nearest image per pair)
                const float4 qh = sh[w][k], ql = sl[w][k];
                float ux = (hi.x - qh.x) + (lo.x - ql.x), uy = (hi.y - qh.y) + (lo.y - ql.y);
                float uz = (hi.z - qh.z) + (lo.z - ql.z);
                const float kx = rintf(ux * iLf), ky = rintf(uy * iLf), kz = rintf(uz * iLf);
                ux = fmaf(-Llo, kx, fmaf(-Lhi, kx, ux));
                uy = fmaf(-Llo, ky, fmaf(-Lhi, ky, uy));
                uz = fmaf(-Llo, kz, fmaf(-Lhi, kz, uz));
                if (fmaf(uz, uz, fmaf(uy, uy, ux * ux)) >= lim) continue;
                const double dx = min_image(xi - sb[w][0][k], L, hL);
                const double dy = min_image(yi - sb[w][1][k], L, hL);
                const double dz = min_image(zi - sb[w][2][k], L, hL);
                const double r2 = dx * dx + dy * dy + dz * dz;
                double gg = 0.0;
                if (r2 < rn2) {
                    const double g1 = exp(-r2 * i2L);
                    gg += g1 * (A2 * g1 + bc * iLam);
                    if (kEnergy) {
                        en += g1 * (S.a * g1 + bc);
                        nn += 1;
                    }
                }
                if (pp && r2 < rc2) {
                    const double r = sqrt(r2);
                    const double ir = 1.0 / r;
                    const double ea = S.alpha * exp(-r * il);
                    gg += ea * ir * ir * (ir + il);
                    if (kEnergy) {
                        ec += ea * ir;
                        nc += 1;
                    }
                }
                fx += gg * dx;
                fy += gg * dy;
                fz += gg * dz;
                if (kEnergy) wv += gg * r2;
            }
        }
    }
    red[w][0][lane] = fx;
    red[w][1][lane] = fy;
    red[w][2][lane] = fz;
    if (kEnergy) {
        const double a0 = warp_sum(valid ? en : 0.0), a1 = warp_sum(valid ? ec : 0.0);
        const double a2 = warp_sum(valid ? wv : 0.0);
        const double a3 = warp_sum(valid ? (double)nn : 0.0), a4 = warp_sum(valid ? (double)nc : 0.0);
        if (lane == 0) {
            ered[w][0] = a0;
            ered[w][1] = a1;
            ered[w][2] = a2;
            ered[w][3] = a3;
            ered[w][4] = a4;
        }
    }
    __syncthreads();
    double* F = S.f64[out_alt ? (st->cur ^ 1) : st->cur];
    if (w == 0) {
        double sx = 0.0, sy = 0.0, sz = 0.0;
        for (int k = 0; k < kFW; ++k) {
            sx += red[k][0][lane];
            sy += red[k][1][lane];
            sz += red[k][2][lane];
        }
        if (chunks == 1) {
            if (valid) {
                F[p] = sx;
                F[N + p] = sy;
                F[2 * N + p] = sz;
                if (!isfinite(sx) || !isfinite(sy) || !isfinite(sz)) atomicOr(&st->error, 1);
            }
        } else {
            // this chunk's partial: slot g * 32 + lane of the chunk's plane
            double* part = E.f64part + (long long)ch * 3 * E.ntiles * kTile;
            const long long k0 = (long long)g * kTile + lane;
            part[k0] = sx;
            part[(long long)E.ntiles * kTile + k0] = sy;
            part[2ll * E.ntiles * kTile + k0] = sz;
        }
        if (kEnergy && lane == 0) {
            double t[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
            for (int k = 0; k < kFW; ++k)
                for (int c = 0; c < 5; ++c) t[c] += ered[k][c];
            // ordered pairs: twice the pairs; this chunk's entries
            long long nent = 0;
            for (int e = ch * kFW; e < e1; e += chunks * kFW) nent += min(kFW, e1 - e);
            add_energy(st, 0.5 * t[0], 0.5 * t[1], 0.5 * t[2], (long long)t[3], (long long)t[4],
                       nent * (kTile * kTile));
        }
    }
    if (chunks == 1) return;
    // the last chunk of tile g to finish adds the partials in chunk order
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(&E.f64cnt[g], 1) == chunks - 1) ? 1 : 0;
    __syncthreads();
    if (!last || w != 0) return;
    __threadfence();
    double sx = 0.0, sy = 0.0, sz = 0.0;
    const long long k0 = (long long)g * kTile + lane, plane = (long long)E.ntiles * kTile;
    for (int c = 0; c < chunks; ++c) {
        const volatile double* part = E.f64part + (long long)c * 3 * plane;
        sx += part[k0];
        sy += part[plane + k0];
        sz += part[2 * plane + k0];
    }
    if (lane == 0) E.f64cnt[g] = 0;
    if (valid) {
        F[p] = sx;
        F[N + p] = sy;
        F[2 * N + p] = sz;
        if (!isfinite(sx) || !isfinite(sy) || !isfinite(sz)) atomicOr(&st->error, 1);
    }
}

}  // namespace

// Clear the energy records before an energy pass.
__global__ void k_ezero(EngineDev E, int only) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= E.nsys || (only >= 0 && s != only)) return;
    for (int k = 0; k < 6; ++k) E.sys[s].st->eacc[k] = 0;
}

namespace {
template <bool kEnergy>
void split_variant(const EngineHost& H, cudaStream_t s, int only, int var, bool gate) {
    const EngineDev& E = H.dev;
    const int nbi = (E.nitems + kForceWarps - 1) / kForceWarps;
    const int g = gate ? 1 : 0;
    if (var == 0) k_force_split<kEnergy, 0><<<nbi, kForceWarps * 32, 0, s>>>(E, only, g);
    else if (var == 1) k_force_split<kEnergy, 1><<<nbi, kForceWarps * 32, 0, s>>>(E, only, g);
    else if (var == 2) k_force_split<kEnergy, 2><<<nbi, kForceWarps * 32, 0, s>>>(E, only, g);
    else k_force_split1<kEnergy><<<E.nitems, 32, 0, s>>>(E, only, g);
}
}  // namespace

void launch_force_pre(const EngineHost& H, cudaStream_t s, bool energy, int only, bool clear) {
    const EngineDev& E = H.dev;
    if (energy && clear) {
        k_ezero<<<(E.nsys + 127) / 128, 128, 0, s>>>(E, only);
        H.count(1);
    }
    H.rec("force", s);
}

void launch_force_variant(const EngineHost& H, cudaStream_t s, bool energy, int only, int var, bool gate) {
    if (energy) split_variant<true>(H, s, only, var, gate);
    else split_variant<false>(H, s, only, var, gate);
    H.count(1);
}

void launch_force_post(const EngineHost& H, cudaStream_t s, bool energy, int only, int out_alt, bool fix) {
    const EngineDev& E = H.dev;
    if (H.precision != 1) {
        const int nb = (E.ntiles + kForceWarps - 1) / kForceWarps;
        if (H.any_verlet) {
            H.rec("force_verlet", s);
            if (energy) k_force_verlet<true><<<E.ntiles, kVW * 32, 0, s>>>(E, only);
            else k_force_verlet<false><<<E.ntiles, kVW * 32, 0, s>>>(E, only);
            H.count(1);
        }
        if (fix) {
            H.rec("force_fix", s);
            k_force_fix<<<nb, kForceWarps * 32, 0, s>>>(E, only, out_alt);
            H.count(1);
        }
    }
    launch_coulomb_pp(H, s, energy, only, out_alt);
}

// A whole force pass outside a step graph: the split kernel runs the variant
// force_unroll fixes, the long one by default (all give the same results).
void launch_force(const EngineHost& H, cudaStream_t s, bool energy, int only, int out_alt) {
    const EngineDev& E = H.dev;
    launch_force_pre(H, s, energy, only);
    if (H.precision == 1) {
        const int ch = E.f64chunks;
        if (energy) k_force_fp64<true><<<E.ntiles * ch, kFW * 32, 0, s>>>(E, only, out_alt, ch);
        else k_force_fp64<false><<<E.ntiles * ch, kFW * 32, 0, s>>>(E, only, out_alt, ch);
        H.count(1);
    } else {
        launch_force_variant(H, s, energy, only, H.fixed_var, false);
    }
    launch_force_post(H, s, energy, only, out_alt);
}

}  // namespace pasta
