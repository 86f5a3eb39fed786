// Integrator and reductions (Sec. II.A): velocity Verlet, box growth of
// Eq. (3) without rescaling positions, isothermal velocity rescale every
// `thermostat_every` steps, FP64 kinetic/potential energy reductions in a
// fixed order, the seeded initial state and steepest-descent relaxation.
//
// Step order (velocity Verlet, then the box grows):
//   k_kick_drift  v += dt/(2M) F;  x += dt v;  wrap into [0, L_n);
//                 displacement and FP32 tile-local coordinates refreshed
//   [rebuild chain if needed]  ->  forces at (x, L_n)
//   k_kick        v += dt/(2M) F;  per-block sum v^2
//   k_finalize    t += dt; step += 1; L = L_base (1 + xi (t - t_base));
//                 thermostat factor when step % thermostat_every == 0
//   k_rescale     v *= factor (when one is pending)
#include "kernels.h"

namespace pasta {

namespace {

struct Slot {
    int s, t, p;
    bool valid;
};

// bx: the block index (a persistent kernel passes the block it plays)
__device__ inline bool slot_of(const EngineDev& E, int only, Slot& o, int bx = blockIdx.x) {
    const int g = bx * kTilesPerBlock + (threadIdx.x >> 5);
    if (g >= E.ntiles) return false;
    const int s = E.tile_sys[g];
    if (s < 0 || (only >= 0 && s != only)) return false;
    const SysConst& S = E.sys[s];
    const int t = g - S.tile_base;
    o.s = s;
    o.t = t;
    o.p = (t < S.T) ? tile_slot0(S, t) + (threadIdx.x & 31) : 0;
    o.valid = (t < S.T) && o.p < tile_end(S, t);
    return true;
}

// Block index of this block within its system (blocks never span systems).
__device__ inline int sys_block(const SysConst& S, int bx = blockIdx.x) {
    return bx - S.tile_base / kTilesPerBlock;
}
__device__ inline int sys_nblocks(const SysConst& S) {
    return (S.T + kTilesPerBlock - 1) / kTilesPerBlock;
}

// Fixed-order block sum of up to 4 doubles into S.blk[blockIdx * 4 + k].
__device__ inline void block_sum4(const SysConst& S, double a, double b, double c, double d) {
    __shared__ double sm[kTilesPerBlock][4];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    d = warp_sum(d);
    if (lane == 0) {
        sm[w][0] = a;
        sm[w][1] = b;
        sm[w][2] = c;
        sm[w][3] = d;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double r = 0.0;
        for (int k = 0; k < kTilesPerBlock; ++k) r += sm[k][threadIdx.x];
        S.blk[4 * sys_block(S) + threadIdx.x] = r;
    }
}

// Fixed-order block sum of one double into S.blk[blockIdx * 4].
__device__ inline void block_sum1(const SysConst& S, double a, int bx = blockIdx.x) {
    __shared__ double sm1[kTilesPerBlock];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    a = warp_sum(a);
    if (lane == 0) sm1[w] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int k = 0; k < kTilesPerBlock; ++k) r += sm1[k];
        S.blk[4 * sys_block(S, bx)] = r;
    }
}

__device__ inline uint64_t splitmix64(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ inline double u01(uint64_t seed, uint64_t k) {
    return __dmul_rn((double)(splitmix64(seed, k) >> 11), 0x1.0p-53);
}

__device__ __forceinline__ double to_double(float f) { return widen(f); }
__device__ __forceinline__ double to_double(double f) { return f; }

template <typename FT>
__device__ inline const FT* cur_force(const SysConst& S, int cur);
template <>
__device__ inline const float* cur_force<float>(const SysConst& S, int cur) { return S.f32[cur]; }
template <>
__device__ inline const double* cur_force<double>(const SysConst& S, int cur) { return S.f64[cur]; }

}  // namespace

// ---------------------------------------------------------------- init
// Slot p = particle p (identity order).  Reading of Sec. III.B: uniform
// positions U(3p+a) L; Box-Muller Gaussians from draws 3N + 2m, 3N + 2m + 1.
__global__ void k_init_rng(EngineDev E, const unsigned long long* seeds) {
    Slot o;
    if (!slot_of(E, -1, o) || !o.valid) return;
    const SysConst& S = E.sys[o.s];
    const int N = S.N, p = o.p;
    const uint64_t seed = seeds[o.s];
    const double L = S.st->L;
    const double sigma = sqrt(S.T_target / S.M);
    const double two_pi = 6.283185307179586;
    for (int a = 0; a < 3; ++a) {
        const uint64_t k = 3ull * p + a;
        S.x[0][a * N + p] = __dmul_rn(u01(seed, k), L);
        const uint64_t m = k / 2;
        const double u1 = u01(seed, 3ull * N + 2 * m);
        const double u2 = u01(seed, 3ull * N + 2 * m + 1);
        const double rad = sqrt(-2.0 * log(1.0 - u1));
        const double ang = __dmul_rn(two_pi, u2);
        const double gz = (k % 2 == 0) ? rad * cos(ang) : rad * sin(ang);
        S.v[0][a * N + p] = __dmul_rn(sigma, gz);
    }
    S.id[0][p] = p;
}

// Per-block sums: mode 0 -> sum v (3 comps), mode 1 -> sum v^2.
__global__ void k_vsum(EngineDev E, int mode, int only) {
    Slot o;
    if (!slot_of(E, only, o)) return;
    const SysConst& S = E.sys[o.s];
    const int c = S.st->cur, N = S.N, p = o.p;
    double a = 0, b = 0, d = 0;
    if (o.valid) {
        const double vx = S.v[c][p], vy = S.v[c][N + p], vz = S.v[c][2 * N + p];
        if (mode == 0) {
            a = vx; b = vy; d = vz;
        } else {
            a = vx * vx + vy * vy + vz * vz;
        }
    }
    block_sum4(S, a, b, d, 0.0);
}

constexpr int kRed = 256;   // threads of the per-system reduction blocks

// Fixed-order block sum (kRed threads): strided partials, then a tree.
__device__ inline double block_sum(double v) {
    __shared__ double sm[kRed / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sm[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = lane < kRed / 32 ? sm[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;   // valid in thread 0
}

// One block per system: fixed-order sum of the system's block partials.
__device__ inline double sys_sum(const SysConst& S, int k) {
    double r = 0.0;
    const int nb = sys_nblocks(S);
    for (int b = threadIdx.x; b < nb; b += kRed) r += S.blk[4 * b + k];
    return block_sum(r);
}

// Remove the centre-of-mass velocity (mode 0) or set the rescale factor
// to reach KE = 3/2 N T (mode 1).
__global__ void k_init_fix(EngineDev E, int mode) {
    const int s = blockIdx.x;
    const SysConst& S = E.sys[s];
    SysState* st = S.st;
    const int lane = threadIdx.x;
    if (mode == 0) {
        const double sx = sys_sum(S, 0), sy = sys_sum(S, 1), sz = sys_sum(S, 2);
        if (lane == 0) {
            st->scratch[0] = sx / S.N;
            st->scratch[1] = sy / S.N;
            st->scratch[2] = sz / S.N;
        }
    } else {
        const double v2 = sys_sum(S, 0);
        if (lane == 0) {
            const double ke = 0.5 * S.M * v2;
            st->vscale = ke > 0.0 ? sqrt(1.5 * (double)S.N * S.T_target / ke) : 0.0;
            st->KE = ke * st->vscale * st->vscale;
        }
    }
}

__global__ void k_sub_com(EngineDev E) {
    Slot o;
    if (!slot_of(E, -1, o) || !o.valid) return;
    const SysConst& S = E.sys[o.s];
    const SysState* st = S.st;
    const int N = S.N, p = o.p;
    S.v[0][p] -= st->scratch[0];
    S.v[0][N + p] -= st->scratch[1];
    S.v[0][2 * N + p] -= st->scratch[2];
}

// Pending thermostat factor on v; with the affine option, the pending box
// factor on x (displacement and tile-frame positions follow).  Launched with
// a small grid that strides over the blocks of slots: on most steps no system
// has a factor pending and every thread returns after reading the flags.
// b0, stride: the blocks of slots this block takes (grid-stride loop)
__device__ __forceinline__ void rescale_body(const EngineDev& E, int only, int b0, int stride) {
    bool any = false;
    for (int s = 0; s < E.nsys; ++s) {
        const SysState* st = E.sys[s].st;
        any |= (st->vscale != 1.0) || (st->xscale != 1.0);
    }
    if (!any) return;
    const int nb = (E.ntiles + kTilesPerBlock - 1) / kTilesPerBlock;
    for (int b = b0; b < nb; b += stride) {
        const int g = b * kTilesPerBlock + (threadIdx.x >> 5);
        if (g >= E.ntiles) continue;
        const int s = E.tile_sys[g];
        if (s < 0 || (only >= 0 && s != only)) continue;
        const SysConst& S = E.sys[s];
        const int t = g - S.tile_base;
        if (t >= S.T) continue;
        const int p = tile_slot0(S, t) + (threadIdx.x & 31);
        if (p >= tile_end(S, t)) continue;
        const SysState* st = S.st;
        const double f = st->vscale, gx = st->xscale;
        const int c = st->cur, N = S.N;
        if (f != 1.0) {
            S.v[c][p] *= f;
            S.v[c][N + p] *= f;
            S.v[c][2 * N + p] *= f;
        }
        if (gx != 1.0) {
            const float4 prev = S.xhi[t * kTile + (threadIdx.x & 31)];
            double xs[3];
            for (int a = 0; a < 3; ++a) {
                const double x0 = S.x[c][a * N + p];
                xs[a] = x0 * gx;
                S.x[c][a * N + p] = xs[a];
                S.disp[a * N + p] += (float)(xs[a] - x0);
            }
            write_xt_moved(S, t, threadIdx.x & 31, xs, st->L, narrow_trunc(st->L), prev);
        }
    }
}

__global__ void k_rescale(EngineDev E, int only) {
    griddep_wait();
    rescale_body(E, only, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------- relax
// Steepest descent (reading of the paper's equilibration from random
// positions): x += gamma F, |dx| clamped to dmax, wrapped.
template <typename FT>
__global__ void k_sd_update(EngineDev E) {
    Slot o;
    if (!slot_of(E, -1, o)) return;     // whole block: systems start on block boundaries
    const SysConst& S = E.sys[o.s];
    SysState* st = S.st;
    const int lane = threadIdx.x & 31;
    float d2 = 0.0f;
    if (o.valid) {
        const int c = st->cur, N = S.N, p = o.p;
        const FT* F = cur_force<FT>(S, c);
        double d[3];
        for (int a = 0; a < 3; ++a) d[a] = S.relax_gamma * to_double(F[a * N + p]);
        const double m = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (m > S.relax_dmax) {
            const double sc = S.relax_dmax / m;
            for (int a = 0; a < 3; ++a) d[a] *= sc;
        }
        const double L = st->L;
        const float4 prev = S.xhi[o.t * kTile + lane];
        double xs[3];
        for (int a = 0; a < 3; ++a) {
            xs[a] = wrap_box_bits(S.x[c][a * N + p] + d[a], L);
            S.x[c][a * N + p] = xs[a];
            const float dd = S.disp[a * N + p] + narrow_trunc(d[a]);
            S.disp[a * N + p] = dd;
            d2 = fmaf(dd, dd, d2);
        }
        write_xt_moved(S, o.t, lane, xs, L, narrow_trunc(L), prev);
    }
    d2 = warp_max(d2);
    block_atomic_max(&st->maxdisp2, d2);
}

// ---------------------------------------------------------------- Verlet
template <typename FT>
__device__ __forceinline__ void kick_drift_body(const EngineDev& E, int bx) {
    Slot o;
    if (!slot_of(E, -1, o, bx)) return;     // whole block: systems start on block boundaries
    const SysConst& S = E.sys[o.s];
    SysState* st = S.st;
    const int lane = threadIdx.x & 31;
    float d2 = 0.0f;
    if (o.valid) {
        const int c = st->cur, N = S.N, p = o.p;
        const FT* F = cur_force<FT>(S, c);
        const double h = S.hkick, dt = S.dt, L = st->L;
        const float4 prev = S.xhi[o.t * kTile + lane];
        double xs[3];
        for (int a = 0; a < 3; ++a) {
            const double v = fma(h, to_double(F[a * N + p]), S.v[c][a * N + p]);
            S.v[c][a * N + p] = v;
            xs[a] = wrap_box_bits(fma(dt, v, S.x[c][a * N + p]), L);
            S.x[c][a * N + p] = xs[a];
            // displacement estimate in FP32 (the list margin covers its rounding)
            const float dd = fmaf(S.dtf, narrow_trunc(v), S.disp[a * N + p]);
            S.disp[a * N + p] = dd;
            d2 = fmaf(dd, dd, d2);
        }
        write_xt_moved(S, o.t, lane, xs, L, narrow_trunc(L), prev);
    }
    d2 = warp_max(d2);
    block_atomic_max(&st->maxdisp2, d2);
}

template <typename FT>
__global__ void k_kick_drift(EngineDev E) {
    griddep_wait();
    kick_drift_body<FT>(E, blockIdx.x);
}

template <typename FT>
__global__ void k_kick(EngineDev E) {
    griddep_wait();
    Slot o;
    if (!slot_of(E, -1, o)) return;
    const SysConst& S = E.sys[o.s];
    const SysState* st = S.st;
    double v2 = 0.0;
    if (o.valid) {
        const int c = st->cur, N = S.N, p = o.p;
        const FT* F = cur_force<FT>(S, c);
        const double h = S.hkick;
        for (int a = 0; a < 3; ++a) {
            const double v = fma(h, to_double(F[a * N + p]), S.v[c][a * N + p]);
            S.v[c][a * N + p] = v;
            v2 = fma(v, v, v2);
        }
    }
    block_sum1(S, v2);
}

// The closing half-kick fused with the conversion of the split force pass's
// fixed-point accumulators (what k_force_fix does, in the same arithmetic):
// F = FP32(facc) 2^-32 is stored for the next step's first half-kick and for
// readers of the state, the accumulators are cleared, v += dt/(2M) F.  Its
// start also closes the force pass's duration for the device tuner.
__device__ __forceinline__ void kick_fix_body(const EngineDev& E, int bx) {
    if (bx == 0 && threadIdx.x == 0) E.tune->t_last = global_ns() - E.tune->t_start;
    Slot o;
    if (!slot_of(E, -1, o, bx)) return;
    const SysConst& S = E.sys[o.s];
    const SysState* st = S.st;
    double v2 = 0.0;
    if (o.valid) {
        const int c = st->cur, N = S.N, p = o.p;
        long long q[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) q[a] = S.facc[a * N + p];
        float* F = S.f32[c];
        const double h = S.hkick;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            S.facc[a * N + p] = 0;
            const float fa = __ll2float_rn(q[a]) * (1.0f / 4294967296.0f);
            F[a * N + p] = fa;
            const double v = fma(h, to_double(fa), S.v[c][a * N + p]);
            S.v[c][a * N + p] = v;
            v2 = fma(v, v, v2);
        }
    }
    block_sum1(S, v2, bx);
}

__global__ void k_kick_fix(EngineDev E) {
    griddep_wait();
    kick_fix_body(E, blockIdx.x);
}

// One block per system.  energy: also record the energy pass's totals.
// Force-pass code variant (ForceTune): account the pass of the step just
// taken (variant tu->cur), then advance the trial: kTuneSteps passes of each
// variant in turn, then keep the fastest.
__device__ inline void tune_step(ForceTune* tu, long long step, bool active) {
    if (!active) return;
    if (tu->phase != 0) {
        const int c = tu->cur;
        tu->acc[c] += (double)tu->t_last;
        tu->n[c] += 1;
        if (tu->n[c] >= kTuneSteps) {
            if (c + 1 < kVariants) {
                tu->cur = c + 1;
                tu->phase = c + 2;
            } else {
                int best = 0;
                for (int k = 1; k < kVariants; ++k)
                    if (tu->acc[k] < tu->acc[best]) best = k;
                tu->cur = best;
                tu->phase = 0;
                tu->trials += 1;
                tu->last_step = step;
            }
        }
    } else if (step >= tu->last_step + kTuneEvery) {
        tu->phase = 1;
        tu->cur = 0;
        for (int k = 0; k < kVariants; ++k) {
            tu->n[k] = 0;
            tu->acc[k] = 0.0;
        }
    }
}

__device__ __forceinline__ void finalize_body(const EngineDev& E, int energy, int s) {
    const SysConst& S = E.sys[s];
    SysState* st = S.st;
    const int lane = threadIdx.x;
    const double v2 = sys_sum(S, 0);
    if (lane != 0) return;
    const double u = 1.0 / 4294967296.0;
    const double pn = (double)st->eacc[0] * u, pc = (double)st->eacc[1] * u, w = (double)st->eacc[2] * u;
    const double Lf = st->L;
    st->L_F = Lf;
    st->t = __dadd_rn(st->t, S.dt);
    st->step += 1;
    st->L = __dmul_rn(st->L_base, __dadd_rn(1.0, __dmul_rn(st->xi_dot, __dsub_rn(st->t, st->t_base))));
    st->xscale = S.affine ? st->L / Lf : 1.0;
    double ke = 0.5 * S.M * v2;
    double f = 1.0;
    if (S.thermostat_every > 0 && (st->step % S.thermostat_every) == 0 && ke > 0.0) {
        f = sqrt(1.5 * (double)S.N * S.T_target / ke);
        ke *= f * f;
    }
    st->vscale = f;
    if (energy) {
        st->KE = ke;
        st->PE_nuc = pn;
        st->PE_coul = pc;
        st->virial = w;
        st->e_L = Lf;
        st->e_t = st->t;
        st->e_step = st->step;
        st->e_pairs_nuc = st->eacc[3] / 2;
        st->e_pairs_coul = st->eacc[4] / 2;
        st->e_cand = st->eacc[5] / 2;
        st->have_energy = 1;
    }
    if (s == 0 && E.tune) tune_step(E.tune, st->step, E.tune_variants && S.force_unroll == 0 && S.list_kind == 0);
}

__global__ void k_finalize(EngineDev E, int energy) {
    griddep_wait();
    finalize_body(E, energy, blockIdx.x);
}

// Energies at the current state (md_energy): KE from the block partials of
// k_vsum(mode 1), PE from the record of an energy force pass.
__global__ void k_energy_now(EngineDev E, int only, double* out) {
    const int s = blockIdx.x;
    if (only >= 0 && s != only) return;
    const SysConst& S = E.sys[s];
    const SysState* st = S.st;
    const int lane = threadIdx.x;
    const double v2 = sys_sum(S, 0);
    if (lane == 0) {
        const double u = 1.0 / 4294967296.0;
        out[0] = 0.5 * S.M * v2;
        out[1] = (double)st->eacc[0] * u;
        out[2] = (double)st->eacc[1] * u;
        out[3] = (double)st->eacc[2] * u;
        out[4] = st->L;
        out[5] = st->t;
        out[6] = (double)st->step;
        out[7] = (double)(st->eacc[3] / 2);
        out[8] = (double)(st->eacc[4] / 2);
    }
}

// ---------------------------------------------------------------- exchange
// Gather current state to original particle order (AoS [N][3]).
template <typename FT>
__global__ void k_gather(EngineDev E, int only, double* ox, double* ov, double* of, int8_t* otype) {
    Slot o;
    if (!slot_of(E, only, o) || !o.valid) return;
    const SysConst& S = E.sys[o.s];
    const SysState* st = S.st;
    const int c = st->cur, N = S.N, p = o.p;
    const int i = S.id[c][p];
    const FT* F = cur_force<FT>(S, c);
    for (int a = 0; a < 3; ++a) {
        if (ox) ox[3 * i + a] = S.x[c][a * N + p];
        if (ov) ov[3 * i + a] = S.v[c][a * N + p];
        if (of) of[3 * i + a] = (double)F[a * N + p];
    }
    if (otype) otype[i] = (int8_t)(i < S.Np ? 1 : 0);
}

// Load a caller state (AoS, original order) into slot order = identity.
__global__ void k_scatter_state(EngineDev E, int only, const double* ix, const double* iv) {
    Slot o;
    if (!slot_of(E, only, o) || !o.valid) return;
    const SysConst& S = E.sys[o.s];
    const SysState* st = S.st;
    const int N = S.N, p = o.p;
    const double L = st->L;
    for (int a = 0; a < 3; ++a) {
        S.x[0][a * N + p] = wrap_box(ix[3 * p + a], L);
        S.v[0][a * N + p] = iv[3 * p + a];
        S.disp[a * N + p] = 0.0f;
    }
    S.id[0][p] = p;
}

// A loaded state (AoS, original order) placed in the current slot order:
// slot p takes particle id[p].  Its displacement since the last rebuild grows
// by the move from the position it replaces (nearest image), and the maximum
// goes to the rebuild decision that follows, so the tiles and lists are kept
// while the rebuild rule allows it (a state saved from this system and loaded
// back keeps them).  With another box side than the current one (Lnew) the
// rebuild is forced.
__global__ void k_load_sorted(EngineDev E, int only, const double* ix, const double* iv, double Lnew) {
    Slot o;
    if (!slot_of(E, only, o)) return;        // whole block: systems start on block boundaries
    const SysConst& S = E.sys[o.s];
    SysState* st = S.st;
    const int lane = threadIdx.x & 31;
    const double L = st->L;
    const bool same_box = Lnew == L;
    float d2 = 0.0f;
    if (o.valid) {
        const int c = st->cur, N = S.N, p = o.p;
        const int i = S.id[c][p];
        const float4 prev = S.xhi[o.t * kTile + lane];
        double xs[3];
        for (int a = 0; a < 3; ++a) {
            const double xn = wrap_box(ix[3 * i + a], Lnew);
            double d = xn - S.x[c][a * N + p];
            if (d > 0.5 * Lnew) d -= Lnew;
            else if (d < -0.5 * Lnew) d += Lnew;
            const float dd = S.disp[a * N + p] + (float)d;
            S.disp[a * N + p] = dd;
            d2 = fmaf(dd, dd, d2);
            S.x[c][a * N + p] = xn;
            S.v[c][a * N + p] = iv[3 * i + a];
            xs[a] = xn;
        }
        if (same_box) write_xt_moved(S, o.t, lane, xs, L, narrow_trunc(L), prev);
    }
    d2 = warp_max(d2);
    block_atomic_max(&st->maxdisp2, d2);
    if (!same_box && threadIdx.x == 0) st->force_rebuild = 1;
}

// Load caller forces (AoS, original order) into the cached force array of
// the current slot order (after the rebuild that follows a loaded state):
// slot p holds particle id[p].
template <typename FT>
__global__ void k_scatter_forces(EngineDev E, int only, const double* f) {
    Slot o;
    if (!slot_of(E, only, o) || !o.valid) return;
    const SysConst& S = E.sys[o.s];
    const int c = S.st->cur, N = S.N, p = o.p;
    const int i = S.id[c][p];
    FT* F = const_cast<FT*>(cur_force<FT>(S, c));
    for (int a = 0; a < 3; ++a) F[a * N + p] = (FT)f[3 * i + a];
}

// Clock and bookkeeping of a loaded state: d_clock = {L, L_base, t, t_base,
// xi_dot, step, L_F}.  Slot order becomes the identity; forces are stale.
// keep_tiles: the state was loaded into the current slot order (k_load_sorted)
// and the rebuild rule decides; otherwise it sits in the original order and a
// rebuild follows.
__global__ void k_set_clock(EngineDev E, int only, const double* c, int keep_tiles) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= E.nsys || (only >= 0 && s != only)) return;
    SysState* st = E.sys[s].st;
    st->L = c[0];
    st->L_base = c[1];
    st->t = c[2];
    st->t_base = c[3];
    st->xi_dot = c[4];
    st->step = (int64_t)c[5];
    st->L_F = c[6];
    st->vscale = 1.0;
    st->xscale = 1.0;
    st->have_energy = 0;
    if (!keep_tiles) {
        st->cur = 0;
        st->cur_next = 0;
        st->force_rebuild = 1;
        st->maxdisp2 = 0u;
        st->last_build = st->step;
    }
}

// The cached forces were just re-evaluated at the current box side (a
// refresh outside a step): record it as their box side L_F.
__global__ void k_mark_forces(EngineDev E, int only) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= E.nsys || (only >= 0 && s != only)) return;
    SysState* st = E.sys[s].st;
    st->L_F = st->L;
}

// Re-base Eq. (3) at the current time when the expansion rate changes.
__global__ void k_set_rate(EngineDev E, int only, double xi) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= E.nsys || (only >= 0 && s != only)) return;
    SysState* st = E.sys[s].st;
    if (st->xi_dot != xi) {
        st->L_base = st->L;
        st->t_base = st->t;
        st->xi_dot = xi;
    }
}

// ---------------------------------------------------------------- launchers
static inline int nblk(const EngineDev& E) { return (E.ntiles + kTilesPerBlock - 1) / kTilesPerBlock; }

void launch_init(const EngineHost& H, cudaStream_t s, const unsigned long long* d_seeds) {
    const EngineDev& E = H.dev;
    k_init_rng<<<nblk(E), kBlock, 0, s>>>(E, d_seeds);
    k_vsum<<<nblk(E), kBlock, 0, s>>>(E, 0, -1);
    k_init_fix<<<E.nsys, kRed, 0, s>>>(E, 0);
    k_sub_com<<<nblk(E), kBlock, 0, s>>>(E);
    k_vsum<<<nblk(E), kBlock, 0, s>>>(E, 1, -1);
    k_init_fix<<<E.nsys, kRed, 0, s>>>(E, 1);
    k_rescale<<<nblk(E), kBlock, 0, s>>>(E, -1);
    H.count(7);
}

void launch_sd_update(const EngineHost& H, cudaStream_t s) {
    const EngineDev& E = H.dev;
    H.rec("sd_update", s);
    if (H.precision == 1) k_sd_update<double><<<nblk(E), kBlock, 0, s>>>(E);
    else k_sd_update<float><<<nblk(E), kBlock, 0, s>>>(E);
    H.count(1);
}

void launch_kick_drift(const EngineHost& H, cudaStream_t s) {
    const EngineDev& E = H.dev;
    H.rec("kick_drift", s);
    if (H.precision == 1) launch_dep(k_kick_drift<double>, nblk(E), kBlock, s, E);
    else launch_dep(k_kick_drift<float>, nblk(E), kBlock, s, E);
    H.count(1);
}

void launch_kick_finalize(const EngineHost& H, cudaStream_t s, bool energy, bool fused_fix) {
    const EngineDev& E = H.dev;
    H.rec("kick", s);
    if (H.precision == 1) launch_dep(k_kick<double>, nblk(E), kBlock, s, E);
    else if (fused_fix) launch_dep(k_kick_fix, nblk(E), kBlock, s, E);
    else launch_dep(k_kick<float>, nblk(E), kBlock, s, E);
    H.rec("finalize", s);
    launch_dep(k_finalize, E.nsys, kRed, s, E, energy ? 1 : 0);
    H.rec("rescale", s);
    launch_dep(k_rescale, std::min(nblk(E), 2 * 148), kBlock, s, E, -1);
    H.count(3);
}

void launch_energy_now(const EngineHost& H, cudaStream_t s, int only, double* d_out) {
    const EngineDev& E = H.dev;
    k_vsum<<<nblk(E), kBlock, 0, s>>>(E, 1, only);
    launch_force(H, s, true, only, 1);
    k_energy_now<<<E.nsys, kRed, 0, s>>>(E, only, d_out);
    H.count(2);
}

void launch_gather(const EngineHost& H, cudaStream_t s, int only, double* ox, double* ov, double* of,
                   int8_t* otype) {
    const EngineDev& E = H.dev;
    if (H.precision == 1) k_gather<double><<<nblk(E), kBlock, 0, s>>>(E, only, ox, ov, of, otype);
    else k_gather<float><<<nblk(E), kBlock, 0, s>>>(E, only, ox, ov, of, otype);
    H.count(1);
}

void launch_set_clock(const EngineHost& H, cudaStream_t s, int only, const double* d_clock, bool keep_tiles) {
    const EngineDev& E = H.dev;
    k_set_clock<<<(E.nsys + 127) / 128, 128, 0, s>>>(E, only, d_clock, keep_tiles ? 1 : 0);
    H.count(1);
}

void launch_mark_forces(const EngineHost& H, cudaStream_t s, int only) {
    const EngineDev& E = H.dev;
    k_mark_forces<<<(E.nsys + 127) / 128, 128, 0, s>>>(E, only);
    H.count(1);
}

void launch_set_rate(const EngineHost& H, cudaStream_t s, int only, double xi_dot) {
    const EngineDev& E = H.dev;
    k_set_rate<<<(E.nsys + 127) / 128, 128, 0, s>>>(E, only, xi_dot);
    H.count(1);
}

void launch_scatter_state(const EngineHost& H, cudaStream_t s, int only, const double* ix, const double* iv) {
    const EngineDev& E = H.dev;
    k_scatter_state<<<nblk(E), kBlock, 0, s>>>(E, only, ix, iv);
    H.count(1);
}

void launch_load_sorted(const EngineHost& H, cudaStream_t s, int only, const double* ix, const double* iv,
                        double L) {
    const EngineDev& E = H.dev;
    k_load_sorted<<<nblk(E), kBlock, 0, s>>>(E, only, ix, iv, L);
    H.count(1);
}

void launch_scatter_forces(const EngineHost& H, cudaStream_t s, int only, const double* iforce) {
    const EngineDev& E = H.dev;
    if (H.precision == 1) k_scatter_forces<double><<<nblk(E), kBlock, 0, s>>>(E, only, iforce);
    else k_scatter_forces<float><<<nblk(E), kBlock, 0, s>>>(E, only, iforce);
    H.count(1);
}

}  // namespace pasta
