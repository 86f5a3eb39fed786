// Paper-literal screened Coulomb (coulomb = 2): every proton pair, nearest
// periodic image, no cutoff (Sec. II.A: "no cutoff radius for the Coulomb
// potential"; the paper's GPU evaluates it by an all-pairs "PP" loop,
// Sec. II.B.1).  O(N_p^2) per step.  Runs after the list-based force kernel,
// which then carries the nuclear term only, and adds the Coulomb force,
// energy and virial of each proton.
//
// Block of 4 warps = 4 consecutive target tiles of one system; the block
// stages one source proton tile at a time in shared memory and every warp
// evaluates its 32 targets against the 32 sources.  Split precision: exact
// hi + lo separations, per-pair nearest image with L as an exact FP32 pair;
// FP64 mode: FP64 positions and arithmetic.
#include "kernels.h"

namespace pasta {
namespace {

constexpr int kPW = 4;   // warps per block

__device__ __forceinline__ float ex2_pp(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_pp(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct KahanF {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

template <bool kEnergy>
__global__ void __launch_bounds__(kPW * 32) k_coulomb_pp_split(EngineDev E, int only, int out_alt) {
    __shared__ float4 sh[kTile], sl[kTile];
    const int g0 = blockIdx.x * kPW;
    if (g0 >= E.ntiles) return;
    const int s = E.tile_sys[g0];
    if (s < 0 || (only >= 0 && s != only)) return;
    const SysConst& S = E.sys[s];
    if (S.coulomb != 2) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int I = g0 + w - S.tile_base;
    const bool active = I < S.Tp;
    if (g0 - S.tile_base >= S.Tp) return;      // whole block past the proton tiles
    SysState* st = S.st;
    const double L = st->L;
    const float Lhi = (float)L, Llo = (float)(L - (double)Lhi), iL = (float)(1.0 / L);
    const float kc = (float)(-1.0 / (S.lambda_s * 0.69314718055994530942));
    const float l2a = (float)log2(S.alpha), il = (float)(1.0 / S.lambda_s);
    const int Ic = active ? I : 0;
    const float4 hi = S.xhi[Ic * kTile + lane], lo = S.xlo[Ic * kTile + lane];
    KahanF kx, ky, kz, ke, kw;
    float nc = 0.f;
    for (int J = 0; J < S.Tp; ++J) {
        __syncthreads();
        if (threadIdx.x < kTile) sh[threadIdx.x] = S.xhi[J * kTile + threadIdx.x];
        else if (threadIdx.x < 2 * kTile) sl[threadIdx.x - kTile] = S.xlo[J * kTile + threadIdx.x - kTile];
        __syncthreads();
        if (!active) continue;
        const int nq = min(kTile, S.Np - J * kTile);
        float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f, wv = 0.f;
        for (int k = 0; k < nq; ++k) {
            const float4 q = sh[k], u = sl[k];
            float dx = (hi.x - q.x) + (lo.x - u.x);
            float dy = (hi.y - q.y) + (lo.y - u.y);
            float dz = (hi.z - q.z) + (lo.z - u.z);
            const float mx = rintf(dx * iL), my = rintf(dy * iL), mz = rintf(dz * iL);
            dx = fmaf(-Llo, mx, fmaf(-Lhi, mx, dx));
            dy = fmaf(-Llo, my, fmaf(-Lhi, my, dy));
            dz = fmaf(-Llo, mz, fmaf(-Lhi, mz, dz));
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const float ri = rsqrt_pp(r2);
            const float ea = ex2_pp(fmaf(r2 * ri, kc, l2a));
            const float vc = ea * ri;
            const bool in = r2 > 0.0f;            // every pair but the target itself
            const float fc = in ? vc * ri * (ri + il) : 0.0f;
            fx = fmaf(fc, dx, fx);
            fy = fmaf(fc, dy, fy);
            fz = fmaf(fc, dz, fz);
            if (kEnergy) {
                e += in ? vc : 0.0f;
                wv = fmaf(fc, r2, wv);
                nc += in ? 1.0f : 0.0f;
            }
        }
        kx.add(fx);
        ky.add(fy);
        kz.add(fz);
        if (kEnergy) {
            ke.add(e);
            kw.add(wv);
        }
    }
    if (!active) return;
    const int p = I * kTile + lane;
    const bool valid = p < S.Np;
    const int N = S.N;
    float* F = S.f32[out_alt ? (st->cur ^ 1) : st->cur];
    if (valid) {
        F[p] += kx.s - kx.c;
        F[N + p] += ky.s - ky.c;
        F[2 * N + p] += kz.s - kz.c;
        if (!isfinite(F[p]) || !isfinite(F[N + p]) || !isfinite(F[2 * N + p])) atomicOr(&st->error, 1);
    }
    if (kEnergy) {
        double en = warp_sum(valid ? (double)ke.s - (double)ke.c : 0.0);
        double wv = warp_sum(valid ? (double)kw.s - (double)kw.c : 0.0);
        double cn = warp_sum(valid ? (double)nc : 0.0);
        if (lane == 0) add_energy(st, 0.0, 0.5 * en, 0.5 * wv, 0, (long long)cn, (long long)S.Np * kTile);
    }
}

template <bool kEnergy>
__global__ void __launch_bounds__(kPW * 32) k_coulomb_pp_fp64(EngineDev E, int only, int out_alt) {
    __shared__ double sx[3][kTile];
    const int g0 = blockIdx.x * kPW;
    if (g0 >= E.ntiles) return;
    const int s = E.tile_sys[g0];
    if (s < 0 || (only >= 0 && s != only)) return;
    const SysConst& S = E.sys[s];
    if (S.coulomb != 2) return;
    if (g0 - S.tile_base >= S.Tp) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int I = g0 + w - S.tile_base;
    const bool active = I < S.Tp;
    SysState* st = S.st;
    const double L = st->L, hL = 0.5 * L;
    const int N = S.N;
    const double* x = S.x[st->cur];
    const int p = (active ? I : 0) * kTile + lane;
    const bool valid = active && p < S.Np;
    const double xi = valid ? x[p] : 0.0, yi = valid ? x[N + p] : 0.0, zi = valid ? x[2 * N + p] : 0.0;
    double fx = 0, fy = 0, fz = 0, en = 0, wv = 0;
    int nc = 0;
    for (int J = 0; J < S.Tp; ++J) {
        __syncthreads();
        if (threadIdx.x < kTile) {
            const int q = J * kTile + threadIdx.x;
            const bool qv = q < S.Np;
            sx[0][threadIdx.x] = qv ? x[q] : 0.0;
            sx[1][threadIdx.x] = qv ? x[N + q] : 0.0;
            sx[2][threadIdx.x] = qv ? x[2 * N + q] : 0.0;
        }
        __syncthreads();
        if (!valid) continue;
        const int nq = min(kTile, S.Np - J * kTile);
        for (int k = 0; k < nq; ++k) {
            if (J * kTile + k == p) continue;
            const double dx = min_image(xi - sx[0][k], L, hL);
            const double dy = min_image(yi - sx[1][k], L, hL);
            const double dz = min_image(zi - sx[2][k], L, hL);
            const double r2 = dx * dx + dy * dy + dz * dz;
            const double r = sqrt(r2);
            const double ea = S.alpha * exp(-r / S.lambda_s);
            const double g = ea * (1.0 / (r2 * r) + 1.0 / (S.lambda_s * r2));
            fx += g * dx;
            fy += g * dy;
            fz += g * dz;
            if (kEnergy) {
                en += ea / r;
                wv += g * r2;
                nc += 1;
            }
        }
    }
    if (!active) return;
    double* F = S.f64[out_alt ? (st->cur ^ 1) : st->cur];
    if (valid) {
        F[p] += fx;
        F[N + p] += fy;
        F[2 * N + p] += fz;
        if (!isfinite(F[p]) || !isfinite(F[N + p]) || !isfinite(F[2 * N + p])) atomicOr(&st->error, 1);
    }
    if (kEnergy) {
        en = warp_sum(valid ? en : 0.0);
        wv = warp_sum(valid ? wv : 0.0);
        const double cn = warp_sum(valid ? (double)nc : 0.0);
        if (lane == 0) add_energy(st, 0.0, 0.5 * en, 0.5 * wv, 0, (long long)cn, (long long)S.Np * kTile);
    }
}

}  // namespace

void launch_coulomb_pp(const EngineHost& H, cudaStream_t s, bool energy, int only, int out_alt) {
    if (!H.any_pp) return;
    const EngineDev& E = H.dev;
    const int nb = (E.ntiles + kPW - 1) / kPW;
    H.rec("coulomb_pp", s);
    if (H.precision == 1) {
        if (energy) k_coulomb_pp_fp64<true><<<nb, kPW * 32, 0, s>>>(E, only, out_alt);
        else k_coulomb_pp_fp64<false><<<nb, kPW * 32, 0, s>>>(E, only, out_alt);
    } else {
        if (energy) k_coulomb_pp_split<true><<<nb, kPW * 32, 0, s>>>(E, only, out_alt);
        else k_coulomb_pp_split<false><<<nb, kPW * 32, 0, s>>>(E, only, out_alt);
    }
    H.count(1);
}

}  // namespace pasta
