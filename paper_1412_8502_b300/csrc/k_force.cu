// Pair forces of Eq. (1) (Sec. II.A): nuclear term for every pair inside
// r_nuc, screened Coulomb for proton pairs inside r_C, nearest periodic
// image, no Newton's-third-law sharing (each target sums over all its
// sources, as the paper's GPU kernel also does, Sec. II.B.1).
//
// Work unit: one warp per 32-particle target tile; the warp walks the tile's
// pair list (tiles whose boxes come within range + skin).  For each source
// tile the 32 source coordinates are staged in shared memory and broadcast
// to all lanes (one LDS.128 per pair step); each lane accumulates the force
// on its own target in registers.  The list is species-sorted by tile, so
// the pair class (pp with/without the nuclear term, like-species nuclear,
// unlike-species nuclear) is warp-uniform per source tile.
//
// Split precision: the FP64 difference of tile origins (computed per list
// entry, one entry per lane) plus FP32 tile-local coordinates give each
// pair separation with an absolute error of a few 1e-7 fm independent of
// the box size; pair arithmetic and per-target accumulation are FP32;
// per-tile energy partials are combined in FP64.
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

enum PairClass { kPPNuc = 0, kPPCoul = 1, kNucSame = 2, kNucCross = 3 };

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
    float Lf, iLf;           // box side for the per-pair image (small boxes)
};

struct Acc {
    float fx, fy, fz;
    float en, ec, w;
    int nn, nc;              // in-range pairs (energy pass only)
};

template <int kClass, bool kSelf, bool kWrap, bool kEnergy>
__device__ __forceinline__ void pair_block(const float4* __restrict__ sj, float tx, float ty, float tz,
                                           const PairConsts& C, Acc& acc) {
    const float S = (kClass == kNucCross) ? C.Scross : C.Ssame;
    const float bS = (kClass == kNucCross) ? C.bcross : C.bsame;
#pragma unroll 8
    for (int k = 0; k < kTile; ++k) {
        const float4 q = sj[k];
        float dx = tx - q.x, dy = ty - q.y, dz = tz - q.z;
        if (kWrap) {
            dx = fmaf(-C.Lf, rintf(dx * C.iLf), dx);
            dy = fmaf(-C.Lf, rintf(dy * C.iLf), dy);
            dz = fmaf(-C.Lf, rintf(dz * C.iLf), dz);
        }
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        float fr = 0.0f;
        if (kClass != kPPCoul) {
            const float gq = ex2_approx(r2 * C.kq);
            const float fn = gq * fmaf(C.A2, gq, S);
            bool in = r2 < C.rn2;
            if (kSelf) in = in && (r2 > 0.0f);
            fr = in ? fn : 0.0f;
            if (kEnergy) {
                acc.en += in ? gq * fmaf(C.a, gq, bS) : 0.0f;
                acc.nn += in ? 1 : 0;
            }
        }
        if (kClass == kPPNuc || kClass == kPPCoul) {
            const float ri = rsqrt_approx(r2);
            const float r = r2 * ri;
            const float ea = ex2_approx(fmaf(r, C.kc, C.l2a));     // alpha e^{-r/lambda}
            const float fc = ea * (ri * ri) * (ri + C.il);
            bool in = r2 < C.rc2;
            if (kSelf) in = in && (r2 > 0.0f);
            fr += in ? fc : 0.0f;
            if (kEnergy) {
                acc.ec += in ? ea * ri : 0.0f;
                acc.nc += in ? 1 : 0;
            }
        }
        acc.fx = fmaf(fr, dx, acc.fx);
        acc.fy = fmaf(fr, dy, acc.fy);
        acc.fz = fmaf(fr, dz, acc.fz);
        if (kEnergy) acc.w = fmaf(fr, r2, acc.w);
    }
}

template <bool kWrap, bool kEnergy>
__device__ __forceinline__ void dispatch(int cls, bool self, const float4* sj, float tx, float ty, float tz,
                                         const PairConsts& C, Acc& acc) {
    if (self) {
        switch (cls) {
            case kPPNuc: pair_block<kPPNuc, true, kWrap, kEnergy>(sj, tx, ty, tz, C, acc); break;
            case kPPCoul: pair_block<kPPCoul, true, kWrap, kEnergy>(sj, tx, ty, tz, C, acc); break;
            case kNucSame: pair_block<kNucSame, true, kWrap, kEnergy>(sj, tx, ty, tz, C, acc); break;
            default: pair_block<kNucCross, true, kWrap, kEnergy>(sj, tx, ty, tz, C, acc); break;
        }
    } else {
        switch (cls) {
            case kPPNuc: pair_block<kPPNuc, false, kWrap, kEnergy>(sj, tx, ty, tz, C, acc); break;
            case kPPCoul: pair_block<kPPCoul, false, kWrap, kEnergy>(sj, tx, ty, tz, C, acc); break;
            case kNucSame: pair_block<kNucSame, false, kWrap, kEnergy>(sj, tx, ty, tz, C, acc); break;
            default: pair_block<kNucCross, false, kWrap, kEnergy>(sj, tx, ty, tz, C, acc); break;
        }
    }
}

struct Kahan {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

constexpr int kForceWarps = 4;   // warps (target tiles) per block

template <bool kWrap, bool kEnergy>
__device__ __forceinline__ void force_tile(const SysConst& S, int I, int out_alt) {
    __shared__ float4 sbuf[kForceWarps][kTile];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float4* sj = sbuf[w];
    SysState* st = S.st;
    const double L = st->L, hL = 0.5 * L;

    PairConsts C;
    C.rn2 = (float)(S.r_nuc * S.r_nuc);
    C.rc2 = S.coulomb ? (float)(S.r_C * S.r_C) : 0.0f;
    C.kq = (float)(-1.0 / (2.0 * S.Lambda * 0.69314718055994530942));
    C.A2 = (float)(2.0 * S.a / S.Lambda);
    C.a = (float)S.a;
    C.Ssame = (float)((S.b + S.c) / S.Lambda);
    C.Scross = (float)((S.b - S.c) / S.Lambda);
    C.bsame = (float)(S.b + S.c);
    C.bcross = (float)(S.b - S.c);
    C.kc = (float)(-1.0 / (S.lambda_s * 0.69314718055994530942));
    C.l2a = (float)log2(S.alpha);
    C.il = (float)(1.0 / S.lambda_s);
    C.Lf = (float)L;
    C.iLf = (float)(1.0 / L);

    const float4 me = S.tpos[I * kTile + lane];
    const double oIx = S.torg[3 * I], oIy = S.torg[3 * I + 1], oIz = S.torg[3 * I + 2];
    const bool Ip = I < S.Tp;
    const int e0 = S.lstart[I], e1 = S.lstart[I + 1];

    Acc acc{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0, 0};
    Kahan ken, kec, kw;
    int nn = 0, nc = 0;

    for (int base = e0; base < e1; base += 32) {
        const int n = min(32, e1 - base);
        const int ent = lane < n ? S.list[base + lane] : 0;
        const int J = ent & (kNucBit - 1);
        float ax = 0.f, ay = 0.f, az = 0.f;
        if (lane < n) {
            ax = (float)min_image(oIx - S.torg[3 * J], L, hL);
            ay = (float)min_image(oIy - S.torg[3 * J + 1], L, hL);
            az = (float)min_image(oIz - S.torg[3 * J + 2], L, hL);
        }
        int Jn = __shfl_sync(0xffffffffu, J, 0);
        float4 qn = S.tpos[Jn * kTile + lane];
        for (int k = 0; k < n; ++k) {
            const int Jk = Jn;
            const int ek = __shfl_sync(0xffffffffu, ent, k);
            const float dxo = __shfl_sync(0xffffffffu, ax, k);
            const float dyo = __shfl_sync(0xffffffffu, ay, k);
            const float dzo = __shfl_sync(0xffffffffu, az, k);
            __syncwarp();
            sj[lane] = qn;
            __syncwarp();
            if (k + 1 < n) {
                Jn = __shfl_sync(0xffffffffu, J, k + 1);
                qn = S.tpos[Jn * kTile + lane];
            }
            const float tx = me.x + dxo, ty = me.y + dyo, tz = me.z + dzo;
            const bool Jp = Jk < S.Tp;
            int cls;
            if (Ip && Jp) cls = S.coulomb ? ((ek & kNucBit) ? kPPNuc : kPPCoul) : kNucSame;
            else cls = (Ip == Jp) ? kNucSame : kNucCross;
            Acc part{acc.fx, acc.fy, acc.fz, 0.f, 0.f, 0.f, 0, 0};
            dispatch<kWrap, kEnergy>(cls, Jk == I, sj, tx, ty, tz, C, part);
            acc.fx = part.fx;
            acc.fy = part.fy;
            acc.fz = part.fz;
            if (kEnergy) {
                ken.add(part.en);
                kec.add(part.ec);
                kw.add(part.w);
                nn += part.nn;
                nc += part.nc;
            }
        }
    }

    const int p = tile_slot0(S, I) + lane;
    const bool valid = p < tile_end(S, I);
    const int N = S.N;
    float* F = S.f32[out_alt ? (st->cur ^ 1) : st->cur];
    if (valid) {
        F[p] = acc.fx;
        F[N + p] = acc.fy;
        F[2 * N + p] = acc.fz;
        if (!isfinite(acc.fx) || !isfinite(acc.fy) || !isfinite(acc.fz)) atomicOr(&st->error, 1);
    }
    if (kEnergy) {
        double en = valid ? ((double)ken.s - (double)ken.c) : 0.0;
        double ec = valid ? ((double)kec.s - (double)kec.c) : 0.0;
        double wv = valid ? ((double)kw.s - (double)kw.c) : 0.0;
        double cn = valid ? (double)nn : 0.0, cc = valid ? (double)nc : 0.0;
        en = warp_sum(en);
        ec = warp_sum(ec);
        wv = warp_sum(wv);
        cn = warp_sum(cn);
        cc = warp_sum(cc);
        if (lane == 0) {
            S.tile_e[8 * I] = 0.5 * en;
            S.tile_e[8 * I + 1] = 0.5 * ec;
            S.tile_e[8 * I + 2] = 0.5 * wv;
            S.tile_e[8 * I + 3] = cn;
            S.tile_e[8 * I + 4] = cc;
        }
    }
}

template <bool kEnergy>
__global__ void __launch_bounds__(kForceWarps * 32) k_force_split(EngineDev E, int only, int out_alt) {
    const int g = blockIdx.x * kForceWarps + (threadIdx.x >> 5);
    if (g >= E.ntiles) return;
    const int s = E.tile_sys[g];
    if (s < 0 || (only >= 0 && s != only)) return;
    const SysConst& S = E.sys[s];
    const int I = g - S.tile_base;
    if (I >= S.T) return;
    if (S.st->need_wrap) force_tile<true, kEnergy>(S, I, out_alt);
    else force_tile<false, kEnergy>(S, I, out_alt);
}

// ---------------------------------------------------------------- FP64
// Validation mode: FP64 positions, per-pair nearest image, FP64 exp/sqrt.
template <bool kEnergy>
__global__ void __launch_bounds__(kForceWarps * 32) k_force_fp64(EngineDev E, int only, int out_alt) {
    __shared__ double sb[kForceWarps][3][kTile];
    const int g = blockIdx.x * kForceWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (g >= E.ntiles) return;
    const int s = E.tile_sys[g];
    if (s < 0 || (only >= 0 && s != only)) return;
    const SysConst& S = E.sys[s];
    const int I = g - S.tile_base;
    if (I >= S.T) return;
    SysState* st = S.st;
    const double L = st->L, hL = 0.5 * L;
    const int N = S.N;
    const double* x = S.x[st->cur];
    const int p = tile_slot0(S, I) + lane;
    const bool valid = p < tile_end(S, I);
    const double xi = valid ? x[p] : 1e30, yi = valid ? x[N + p] : 1e30, zi = valid ? x[2 * N + p] : 1e30;
    const bool Ip = I < S.Tp;
    const double rn2 = S.r_nuc * S.r_nuc, rc2 = S.r_C * S.r_C;
    const double A2 = 2.0 * S.a / S.Lambda;
    double fx = 0, fy = 0, fz = 0, en = 0, ec = 0, wv = 0;
    int nn = 0, nc = 0;
    const int e0 = S.lstart[I], e1 = S.lstart[I + 1];
    for (int e = e0; e < e1; ++e) {
        const int J = S.list[e] & (kNucBit - 1);
        const int q = tile_slot0(S, J) + lane;
        const bool qv = q < tile_end(S, J);
        __syncwarp();
        sb[w][0][lane] = qv ? x[q] : -1e30;
        sb[w][1][lane] = qv ? x[N + q] : -1e30;
        sb[w][2][lane] = qv ? x[2 * N + q] : -1e30;
        __syncwarp();
        const bool Jp = J < S.Tp;
        const bool pp = Ip && Jp && S.coulomb;
        const double bc = (Ip == Jp) ? (S.b + S.c) : (S.b - S.c);
        for (int k = 0; k < kTile; ++k) {
            if (J == I && k == lane) continue;
            const double dx = min_image(xi - sb[w][0][k], L, hL);
            const double dy = min_image(yi - sb[w][1][k], L, hL);
            const double dz = min_image(zi - sb[w][2][k], L, hL);
            const double r2 = dx * dx + dy * dy + dz * dz;
            double gg = 0.0;
            if (r2 < rn2) {
                const double g1 = exp(-r2 / (2.0 * S.Lambda));
                gg += g1 * (A2 * g1 + bc / S.Lambda);
                if (kEnergy) {
                    en += g1 * (S.a * g1 + bc);
                    nn += 1;
                }
            }
            if (pp && r2 < rc2) {
                const double r = sqrt(r2);
                const double ea = S.alpha * exp(-r / S.lambda_s);
                gg += ea * (1.0 / (r2 * r) + 1.0 / (S.lambda_s * r2));
                if (kEnergy) {
                    ec += ea / r;
                    nc += 1;
                }
            }
            fx += gg * dx;
            fy += gg * dy;
            fz += gg * dz;
            if (kEnergy) wv += gg * r2;
        }
    }
    double* F = S.f64[out_alt ? (st->cur ^ 1) : st->cur];
    if (valid) {
        F[p] = fx;
        F[N + p] = fy;
        F[2 * N + p] = fz;
        if (!isfinite(fx) || !isfinite(fy) || !isfinite(fz)) atomicOr(&st->error, 1);
    }
    if (kEnergy) {
        en = warp_sum(valid ? en : 0.0);
        ec = warp_sum(valid ? ec : 0.0);
        wv = warp_sum(valid ? wv : 0.0);
        const double cn = warp_sum(valid ? (double)nn : 0.0), cc = warp_sum(valid ? (double)nc : 0.0);
        if (lane == 0) {
            S.tile_e[8 * I] = 0.5 * en;
            S.tile_e[8 * I + 1] = 0.5 * ec;
            S.tile_e[8 * I + 2] = 0.5 * wv;
            S.tile_e[8 * I + 3] = cn;
            S.tile_e[8 * I + 4] = cc;
        }
    }
}

}  // namespace

void launch_force(const EngineHost& H, cudaStream_t s, bool energy, int only, int out_alt) {
    const EngineDev& E = H.dev;
    const int nb = (E.ntiles + kForceWarps - 1) / kForceWarps;
    H.rec("force", s);
    if (H.precision == 1) {
        if (energy) k_force_fp64<true><<<nb, kForceWarps * 32, 0, s>>>(E, only, out_alt);
        else k_force_fp64<false><<<nb, kForceWarps * 32, 0, s>>>(E, only, out_alt);
    } else {
        if (energy) k_force_split<true><<<nb, kForceWarps * 32, 0, s>>>(E, only, out_alt);
        else k_force_split<false><<<nb, kForceWarps * 32, 0, s>>>(E, only, out_alt);
    }
    H.count(1);
}

}  // namespace pasta
