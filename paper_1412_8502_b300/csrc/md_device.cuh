// Device-side data layout shared by the kernels of the nucleon MD library.
//
// One "engine" advances one or more independent systems.  Every per-system
// quantity lives in device memory behind a SysConst descriptor; all kernels
// take the descriptor table and work over a global space of 32-particle
// tiles (each system's tiles start at a multiple of kTilesPerBlock, so a
// 256-thread block never spans two systems).
//
// Particle storage is structure-of-arrays in the current spatially sorted
// order: protons occupy sorted slots [0, Np), neutrons [Np, N).  Proton tile
// t covers slots [32 t, 32 t + 32) ∩ [0, Np); neutron tile Tp + u covers
// [Np + 32 u, ...) ∩ [Np, N).  Positions and velocities are FP64 (x[a*N + p]
// is axis a of sorted slot p).  The force kernel reads each position as a
// pair of FP32 numbers, xhi + xlo, of the periodic image nearest its tile's
// origin O_t (fixed at the last pair-list rebuild), refreshed every
// step: xhi[32 t + lane] = xt rounded to 24 significant bits, xlo = the
// remainder rounded to FP32 (|xt - xhi - xlo| <= 2^-49 |xt|).
#pragma once
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

namespace pasta {

struct ClusterBufs;

constexpr int kTile = 32;
constexpr int kTilesPerBlock = 8;
constexpr int kBlock = kTile * kTilesPerBlock;
constexpr float kPad = 1.0e9f;          // local coordinate of an empty slot
// Pair-list entry: bits 0-23 source tile J, 24-29 periodic shift code
// (sx+1) | (sy+1) << 2 | (sz+1) << 4 moving J next to the target tile,
// bit 30 set when the nuclear term is reachable.
constexpr int kJMask = (1 << 24) - 1;
constexpr int kShiftPos = 24;
constexpr int kNucBit = 1 << 30;
constexpr int kShiftNone = 1 | (1 << 2) | (1 << 4);   // shift code of (0, 0, 0)

// Mutable per-system scalars (device memory).
struct SysState {
    double L, L_base, t, t_base, xi_dot;
    double L_F;              // box side of the cached forces
    double L_build;          // box side at the last rebuild
    double KE, PE_nuc, PE_coul, virial;     // last recorded energies
    double e_L, e_t;         // box side / time of the recorded energies
    int64_t e_pairs_nuc, e_pairs_coul;   // in-range pairs i<j of that pass
    int64_t e_cand;                      // candidate pairs evaluated in that pass
    float hsum;              // sum of tile half-extents at the last rebuild
    int pad1;
    double vscale;           // pending thermostat factor (1 = none)
    double xscale;           // pending affine position factor (1 = none)
    int64_t step, last_build, n_rebuilds, e_step;
    int64_t list_total;
    double scratch[3];       // initialisation scratch (centre-of-mass velocity)
    int cur;                 // which x/v/id/f buffer is current
    int cur_next;            // buffer the running rebuild writes
    int rebuild;             // this step rebuilds (set by the decision kernel)
    int force_rebuild;       // rebuild at the next decision regardless
    int pad2;
    int need_wrap;           // per-pair minimum image needed in FP32
    int have_energy;         // energies recorded by a step
    int error;               // bit 0: non-finite force; bit 2: Verlet list pool exhausted
    unsigned maxdisp2;       // float bits of max |disp|^2 since the rebuild
    unsigned hmax;           // float bits of max tile half-extent at rebuild
    int pad0;
    unsigned long long vtop;     // Verlet list pool slots taken at the last rebuild
    unsigned long long vpairs;   // Verlet list entries written at the last rebuild
    // energy record of the running force pass: PE_nuc, PE_coul, virial in
    // 2^-32 MeV fixed point; twice the in-range nuclear / Coulomb pairs and
    // twice the candidate pairs (cleared before each energy pass)
    long long eacc[6];
};

// FP32 constants of the split-precision pair terms, computed on the host
// from the FP64 parameters of the system (pair_consts in engine.cu).
struct PairF {
    float rn2, rc2;          // squared cutoffs (rc2 = 0 unless coulomb == 1)
    float kq;                // -1/(2 Lambda ln 2): g = 2^(r2 kq)
    float A2;                // 2a/Lambda
    float a;                 // a
    float Ssame, Scross;     // (b+c)/Lambda, (b-c)/Lambda
    float bsame, bcross;     // b+c, b-c
    float kc;                // -1/(lambda ln 2)
    float l2a;               // log2(alpha)
    float il;                // 1/lambda
    float Rn2, Rc2;          // source filter radii^2 around the targets' current box: cutoff + 2e-3 fm
};

// Per-system constants and device pointers.
struct SysConst {
    int N, Np, T, Tp;        // particles, protons, tiles, proton tiles
    int tile_base;           // first global tile (multiple of kTilesPerBlock)
    int item_base;           // first global force work item (multiple of 4)
    int n_items;             // force work items: kPChunks per proton tile, kNChunks per neutron tile
    int nbits;               // spatial-sort bits per axis
    long long bin_base;      // first global bin (2 species x 2^(3 nbits) bins)
    long long nbins;         // bins per species
    long long list_cap;      // entries available in `list`
    // physics
    double dt, M, T_target, skin;
    double a, b, c, Lambda, lambda_s, alpha, r_nuc, r_C;
    double r_pp, r_np, relax_gamma, relax_dmax;
    double hkick;            // dt / (2 M): velocity Verlet half kick per unit force
    float dtf;               // dt in FP32 (displacement estimates)
    int thermostat_every, rebuild_every, coulomb, energy_every;
    int affine;              // scale positions with the box (option, not the paper)
    int list_kind;           // 0 half tile-pair lists, 1 per-particle Verlet lists
    int force_unroll;        // split force-pass code variant: 0 automatic, 4 long, 2 compact, 1 minimal
    int uf_limit;            // iterations of a union-find loop before it gives up (cluster analyses)
    PairF pf;
    // state arrays (index [cur] is current)
    double* x[2];
    double* v[2];
    int* id[2];
    float* f32[2];
    double* f64[2];
    float* disp;             // [3N] displacement since the last rebuild
    unsigned* key;           // [N] bin of each slot (rebuild scratch)
    int* slot;               // [N] scatter scratch
    float4* xhi;             // [T*32] FP32 high part of the tile-frame position
    float4* xlo;             // [T*32] FP32 low part (xhi + xlo = position)
    float* torgf;            // [T*4] FP32 origin (x,y,z) and max half-extent
    float* thalf;            // [T*3] tile half-extents at rebuild
    float4* sorg;            // [ceil(T/32)] super-tile (32 tiles) box centre
    float4* shalf;           // [ceil(T/32)] super-tile box half extents
    int* lcount;             // [T] entries per tile
    int* lnear;              // [T] of which near (written from the front of the region)
    int* list;               // [list_cap] tile-pair entries: J | kNucBit
    long long* facc;         // [3N] split precision: forces in 2^-32 MeV/fm fixed point
    // per-particle Verlet lists (list_kind 1): for tile t, lane l's k-th entry
    // is vlist[voff[t] + 32 k + l], k < vcount[32 t + l] <= vwidth[t]; an entry
    // is the source's tile slot (32 J + lane) | shift code | nuclear flag
    int* vlist;              // [vcap]
    int* vcount;             // [T*32]
    long long* voff;         // [T]
    int* vwidth;             // [T]
    long long vcap;          // pool capacity (entries)
    double* blk;             // [T/8 * 4] per-block KE partials
    ClusterBufs* cl;         // cluster-analysis buffers (device struct)
    SysState* st;
};

// Global tables of an engine.
// Choice between the code variants of the split force pass, made on the
// device by timing (the variants give bitwise the same results): every
// kTuneEvery steps kTuneSteps force passes run with each variant, their
// durations (%globaltimer at the start of the force kernel's block 0 to the
// start of the k_force_fix launch that follows it) are summed, and the
// fastest variant is kept until the next trial.  Each variant is its own
// kernel: in a step graph a SWITCH node launches the selected one (k_decide
// sets it); in plain graphs all of them are launched and all but one return at
// once.  The first trial comes at step kTuneEvery: until then the long variant
// runs (systems start dense).  The fourth variant runs the minimal code with
// one warp per block, so that a warp whose work item ends frees its slot
// without waiting for the other warps of a block (faster where items differ
// much in cost, as in clustered states; slower in dense ones, where the four
// adjacent tiles of a block share their source tiles in L1).
constexpr int kTuneEvery = 500;
constexpr int kTuneSteps = 4;
constexpr int kVariants = 4;         // long, compact, minimal, minimal in one-warp blocks
struct ForceTune {
    unsigned long long t_start;  // start of the running force pass, ns
    unsigned long long t_last;   // duration of the last force pass, ns
    int cur;                     // tuner: variant to run next: 0 long, 1 compact, 2 minimal, 3 minimal (one-warp blocks)
    int sel;                     // variant of this step's pass (set by k_decide from cur or force_unroll)
    int phase;                   // 0 idle, 1 + v timing variant v
    int trials;                  // trials completed
    int n[kVariants];
    long long last_step;         // step of system 0 at the last decision (0 before the first)
    double acc[kVariants];       // summed durations per variant, ns
};

// Programmatic dependent launch (launch_dep): wait for the kernel ahead on
// the stream to finish and its writes to be visible (a no-op for a kernel
// launched without the attribute), then let the kernel behind be scheduled
// at once, so that its launch overlaps this one's run (its blocks wait here
// in turn before touching any data).  The first statement of every kernel
// launched with launch_dep.
__device__ __forceinline__ void griddep_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct EngineDev {
    const SysConst* sys;     // [nsys]
    const int* tile_sys;     // [ntiles] global tile -> system (-1: padding)
    const int* item_sys;     // [nitems] global force work item -> system (-1: padding)
    int nitems;              // global force work items (multiple of 4)
    int nsys;
    int ntiles;              // global tiles (multiple of kTilesPerBlock)
    long long nbins_total;   // global bins
    unsigned* hist;          // [nbins_total]
    unsigned* binstart;      // [nbins_total] exclusive scan of hist
    unsigned* cursor;        // [nbins_total] scatter cursors
    unsigned* blocksum;      // [scan blocks]
    int* any_rebuild;        // set when any system rebuilds this step
    unsigned long long* cond_runs;   // step-graph rebuilds run through the conditional node
    ForceTune* tune;                 // force-pass code variant (automatic choice)
    int tune_variants;               // 1: steps select the variant (SWITCH node) and the tuner runs
    // FP64 mode with fewer tiles than SMs: a tile's list entries run in
    // f64chunks blocks whose partial forces meet in f64part ([chunk][3][tile
    // slot]); f64cnt[tile] counts the finished chunks (the last one adds them)
    int f64chunks;
    double* f64part;
    int* f64cnt;
};

// Engines below this many particles run one force-pass variant: the SWITCH
// node costs ~7 us per step, more than the variants gain on short passes.
constexpr long long kVariantMinN = 131072;

// Control block of the persistent step kernel (k_persist.cuh).
struct PersistCtl {
    unsigned bar;                // barrier arrivals of this launch (cleared before it)
    unsigned work;               // next force work item
    int error;                   // 1: a barrier wait gave up (sticky until the host reads it)
    int pad;
};

// Force work items of a system.  A proton tile's list holds its near
// entries (nuclear range) first and its Coulomb-only entries from the back of
// its region; it gives kPChunks items: items 0 .. kPNear-1 equal parts of the
// near entries (item 0 also the tile with itself), the others equal parts of
// the Coulomb-only entries.  A neutron tile gives kNChunks items: in a system
// below kSplitRho the halves of its list (item 0 with the tile itself), in a
// denser one the whole list and an empty item (there neutron tiles are light:
// their entries pass few sources; in clustered, dilute states the tiles inside
// nuclei are among the heaviest items, and halving them shortens the tail of
// the pass).  Items c of kItemGroup adjacent tiles sit side by side (one block
// of the force kernel); proton items come first; with whole neutron lists the
// unused items are the last ones.
constexpr int kPChunks = 4;
constexpr int kPNear = 2;
constexpr int kNChunks = 2;
constexpr double kSplitRho = 0.02;      // fm^-3
constexpr int kItemGroup = 4;
__host__ __device__ inline int proton_items(int Tp) {
    return (Tp + kItemGroup - 1) / kItemGroup * kItemGroup * kPChunks;
}
__host__ __device__ inline int neutron_items(int Tn) {
    return (Tn + kItemGroup - 1) / kItemGroup * kItemGroup * kNChunks;
}
__host__ __device__ inline int sys_items(int T, int Tp) { return proton_items(Tp) + neutron_items(T - Tp); }
__host__ __device__ inline int item_index(const SysConst& s, int t, int c) {
    if (t >= s.Tp) {
        const int u = t - s.Tp;
        return proton_items(s.Tp) + ((u / kItemGroup) * kNChunks + c) * kItemGroup + u % kItemGroup;
    }
    return ((t / kItemGroup) * kPChunks + c) * kItemGroup + t % kItemGroup;
}
// Position in tile I's list region of its e-th entry (near entries first).
__device__ inline int list_pos(const SysConst& s, int e, int nnear) { return e < nnear ? e : s.T - 1 - (e - nnear); }

__host__ __device__ inline int tile_slot0(const SysConst& s, int t) {
    return t < s.Tp ? t * kTile : s.Np + (t - s.Tp) * kTile;
}
__host__ __device__ inline int tile_end(const SysConst& s, int t) {
    return t < s.Tp ? min(s.Np, (t + 1) * kTile) : min(s.N, s.Np + (t - s.Tp + 1) * kTile);
}

// Add a work unit's energies (FP64) and pair counts (twice the pairs) to the
// system's energy record with integer atomics: the totals do not depend on
// the order of the additions.
__device__ inline void add_energy(SysState* st, double pe_nuc, double pe_coul, double vir, long long twice_nn,
                                  long long twice_nc, long long twice_cand) {
    const double k = 4294967296.0;
    atomicAdd((unsigned long long*)&st->eacc[0], (unsigned long long)__double2ll_rn(pe_nuc * k));
    atomicAdd((unsigned long long*)&st->eacc[1], (unsigned long long)__double2ll_rn(pe_coul * k));
    atomicAdd((unsigned long long*)&st->eacc[2], (unsigned long long)__double2ll_rn(vir * k));
    atomicAdd((unsigned long long*)&st->eacc[3], (unsigned long long)twice_nn);
    atomicAdd((unsigned long long*)&st->eacc[4], (unsigned long long)twice_nc);
    atomicAdd((unsigned long long*)&st->eacc[5], (unsigned long long)twice_cand);
}

// error-free a + b = s + e (FP32)
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Move a source (hi + lo) by the periodic shift of a list entry: each axis
// code c in {0, 1, 2} adds (c - 1) L, L = Lhi + Llo, with an error-free sum.
__device__ __forceinline__ void apply_shift(int shk, float Lhi, float Llo, float4& h, float4& l) {
    const float fx = (float)((shk & 3) - 1), fy = (float)(((shk >> 2) & 3) - 1), fz = (float)(((shk >> 4) & 3) - 1);
    float er;
    two_sum_f(h.x, fx * Lhi, h.x, er);
    l.x = l.x + fx * Llo + er;
    two_sum_f(h.y, fy * Lhi, h.y, er);
    l.y = l.y + fy * Llo + er;
    two_sum_f(h.z, fz * Lhi, h.z, er);
    l.z = l.z + fz * Llo + er;
}

// Wrap into [0, L): one period at most (displacements per step << L).
static __host__ __device__ __noinline__ double wrap_box_slow(double x, double L);
__host__ __device__ inline double wrap_box(double x, double L) {
    if (x >= L) {
        x -= L;
    } else if (x < 0.0) {
        x += L;
        if (x >= L) x = 0.0;
    }
    return x;
}

// Nearest image of a difference with |d| < 1.5 L, comparison form.
static __host__ __device__ __noinline__ double wrap_box_slow(double x, double L) { return wrap_box(x, L); }
static __device__ __noinline__ double image_shift(double x, double L, float k) { return x - L * (double)k; }

__device__ inline double min_image(double d, double L, double hL) {
    if (d > hL) d -= L;
    else if (d < -hL) d += L;
    return d;
}

// ---- FP64 state without the FP64 pipe.  On this part FP64 arithmetic and
// every conversion to or from a 64-bit type issue at about 1/64 of the FP32
// rate, so the exact format work around the FP64 state (widening the FP32
// forces, splitting positions into FP32 pairs, range tests) is done with
// integer operations on the IEEE-754 bit patterns.

// Bit patterns of FP32/FP64 values (device intrinsics; memcpy on the host,
// where the helpers below are tested against the hardware conversions).
__host__ __device__ __forceinline__ unsigned f_bits(float f) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    unsigned u;
    memcpy(&u, &f, sizeof u);
    return u;
#endif
}
__host__ __device__ __forceinline__ float f_from(unsigned u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, sizeof f);
    return f;
#endif
}
__host__ __device__ __forceinline__ unsigned long long d_bits(double d) {
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(d);
#else
    unsigned long long u;
    memcpy(&u, &d, sizeof u);
    return u;
#endif
}
__host__ __device__ __forceinline__ double d_from(unsigned long long u) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double d;
    memcpy(&d, &u, sizeof d);
    return d;
#endif
}

// Order-preserving 32-bit key of a float (a < b exactly when key(a) < key(b))
// for integer warp min / max reductions.
__device__ __forceinline__ unsigned fkey(float v) {
    const unsigned b = __float_as_uint(v);
    return (b >> 31) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(unsigned k) {
    return __uint_as_float((k >> 31) ? (k & 0x7fffffffu) : ~k);
}

// The rare cases below go through these out-of-line converters: inlined,
// the compiler predicates them into the common path, where their FP64
// instructions issue for every particle.
static __host__ __device__ __noinline__ double widen_slow(float f) { return (double)f; }
static __host__ __device__ __noinline__ float narrow_slow(double d) { return (float)d; }
static __host__ __device__ __noinline__ float2 split_slow(double x) {
    const float hi = (float)x;
    return make_float2(hi, (float)(x - (double)hi));
}

// Exact (double)f.  Zero and normal f on the integer path; subnormal, inf
// and NaN through the converter.
__host__ __device__ __forceinline__ double widen(float f) {
    const unsigned b = f_bits(f);
    const unsigned a = b & 0x7fffffffu;
    const bool normal = (a - 0x00800000u) < 0x7f000000u;
    if (!normal && a != 0u) return widen_slow(f);
    const unsigned long long mag = normal ? ((unsigned long long)a << 29) + (896ull << 52) : 0ull;
    return d_from(((unsigned long long)(b & 0x80000000u) << 32) | mag);
}

// d truncated to FP32 (|result| <= |d|, relative error below 2^-23) for d
// in the normal FP32 range or zero; other values through the converter.
__host__ __device__ __forceinline__ float narrow_trunc(double d) {
    const unsigned long long b = d_bits(d);
    const unsigned h = (unsigned)(b >> 32);
    const unsigned e = (h >> 20) & 0x7ffu;
    if (e == 0u && (b << 1) == 0ull) return f_from(h & 0x80000000u);
    if (e - 897u >= 254u) return narrow_slow(d);
    return f_from((h & 0x80000000u) | ((e - 896u) << 23) | ((unsigned)(b >> 29) & 0x7fffffu));
}

// x = hi + lo: hi is x rounded to 24 significant bits (to nearest, ties
// away from zero, so |x - hi| <= ulp(hi)/2), lo the remainder rounded to
// FP32 (|x - hi - lo| <= 2^-49 |x|), from integer operations for
// 2^-74 <= |x| < 2^126; other x (zero included) through the converter as
// hi = fp32(x), lo = fp32(x - hi).
__host__ __device__ __forceinline__ void split_hilo(double x, float& hi, float& lo) {
    const unsigned long long b = d_bits(x);
    const unsigned e = (unsigned)(b >> 52) & 0x7ffu;
    if (e - 949u >= 200u) {
        const float2 q = split_slow(x);
        hi = q.x;
        lo = q.y;
        return;
    }
    const unsigned s = (unsigned)(b >> 32) & 0x80000000u;
    // adding half a unit of the 24-bit significand rounds it (a carry may
    // step the exponent, which is the correct rounded value)
    const unsigned long long r = b + (1ull << 28);
    hi = f_from(s | ((((unsigned)(r >> 52) & 0x7ffu) - 896u) << 23) | ((unsigned)(r >> 29) & 0x7fffffu));
    // x - hi in units of 2^(e - 1075), the weight of the last bit of x
    const int low = (int)((unsigned)b & 0x1fffffffu) - (int)(((unsigned)b & 0x10000000u) << 1);
    lo = (float)low * f_from(s | ((e - 948u) << 23));
}

__device__ inline float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ inline double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ inline float warp_max(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Store slot (t, lane)'s tile-frame position xt as the FP32 pair hi + lo
// (empty slots: far away, zero low part).  h.w carries the particle's slot
// index (bit pattern of an int; -1 for an empty slot).
__device__ inline void store_xt(const SysConst& s, int t, int lane, const double* xt, bool valid) {
    float4 h, l;
    h.w = __int_as_float(valid ? tile_slot0(s, t) + lane : -1);
    l.w = 0.0f;
    if (valid) {
        split_hilo(xt[0], h.x, l.x);
        split_hilo(xt[1], h.y, l.y);
        split_hilo(xt[2], h.z, l.z);
    } else {
        h.x = h.y = h.z = kPad;
        l.x = l.y = l.z = 0.0f;
    }
    s.xhi[t * kTile + lane] = h;
    s.xlo[t * kTile + lane] = l;
}

// A particle that moved (by much less than L/2) since its tile-frame
// position was last stored: its new image is the one next to the previous
// one, i.e. xs itself unless the particle crossed a face of the box since
// the last rebuild (then xs - k L, k = +-1, in FP64).  prev: the stored
// high parts; Lf: L truncated to FP32.
__device__ inline void write_xt_moved(const SysConst& s, int t, int lane, const double* xs, double L, float Lf,
                                      const float4& prev) {
    double xt[3] = {xs[0], xs[1], xs[2]};
    const float pv[3] = {prev.x, prev.y, prev.z};
    for (int a = 0; a < 3; ++a) {
        const float d = narrow_trunc(xs[a]) - pv[a];
        if (fabsf(d) > 0.5f * Lf) xt[a] = image_shift(xs[a], L, rintf(d / Lf));
    }
    store_xt(s, t, lane, xt, true);
}

// xs wrapped into [0, L) (x >= L: x - L; x < 0: x + L, or 0 if that rounds
// to L), the common in-range case decided on the bit patterns.
__host__ __device__ __forceinline__ double wrap_box_bits(double x, double L) {
    const long long xb = (long long)d_bits(x);
    if (xb >= 0 && xb < (long long)d_bits(L)) return x;       // 0 <= x < L (L > 0)
    return wrap_box_slow(x, L);
}

// Block-level max of a non-negative float (one value per warp, lane 0
// holding it), then one atomicMax per block.  Every thread of the block
// must call it.
__device__ inline void block_atomic_max(unsigned* addr, float warp_value) {
    __shared__ float sm[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) sm[w] = warp_value;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.0f;
        for (int k = 0; k < nw; ++k) m = fmaxf(m, sm[k]);
        if (m > 0.0f) atomicMax(addr, __float_as_uint(m));
    }
}

// atomicMax on the bit pattern of a non-negative float.
__device__ inline void atomic_max_pos(unsigned* addr, float v) {
    atomicMax(addr, __float_as_uint(fmaxf(v, 0.0f)));
}

}  // namespace pasta
