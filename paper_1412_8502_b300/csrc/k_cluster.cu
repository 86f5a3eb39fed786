// Cluster algorithm of Sec. II.C on the GPU.
//
// Protons closer than r_pp (nearest image) are linked; the connected
// components are the clusters (lock-free union-find with hooking of the
// larger root onto the smaller one).  Each cluster is labelled by its
// smallest original proton index.  A neutron joins the cluster of its
// nearest proton closer than r_np (equal distances: smaller proton index),
// otherwise it is free.  Candidate pairs come from the current tiles: their
// boxes (taken at the last pair-list rebuild) are tested against r + skin,
// which covers every particle's drift since then.  The link and assignment
// decisions are those of FP64 squared distances evaluated as
//   dx = x_i - x_j; nearest image by comparison with L/2;
//   d2 = (dx*dx + dy*dy) + dz*dz        (no fused multiply-add)
// so they are exact and identical to a serial FP64 evaluation.  A pair is
// first screened in FP32 from the exact hi + lo tile-frame positions (the
// separation is exact before rounding, so the FP32 d2 is within a few ulp
// of the FP64 one); only pairs within kBand of the threshold, and every
// neutron-proton candidate inside r_np, are evaluated in FP64.
#include "kernels.h"

namespace pasta {

namespace {

__device__ __forceinline__ double d2_exact(double xi, double yi, double zi, double xj, double yj, double zj,
                                           double L, double hL) {
    double dx = __dsub_rn(xi, xj), dy = __dsub_rn(yi, yj), dz = __dsub_rn(zi, zj);
    if (dx > hL) dx = __dsub_rn(dx, L); else if (dx < -hL) dx = __dadd_rn(dx, L);
    if (dy > hL) dy = __dsub_rn(dy, L); else if (dy < -hL) dy = __dadd_rn(dy, L);
    if (dz > hL) dz = __dsub_rn(dz, L); else if (dz < -hL) dz = __dadd_rn(dz, L);
    double s = __dmul_rn(dx, dx);
    s = __dadd_rn(s, __dmul_rn(dy, dy));
    s = __dadd_rn(s, __dmul_rn(dz, dz));
    return s;
}

// Roots only ever hook onto smaller roots and path halving only shortens
// paths, so every walk ends.  Each loop is bounded all the same by the
// host-set limit (md_params.uf_iter_limit); a loop that reaches it gives up
// and records the fact in *gave_up (ClusterBufs.stats[7], cleared by the
// init kernels), which the host reports as MD_ETIMEOUT.  A walk that gives
// up returns the slot it reached, a valid index, so nothing downstream
// reads out of bounds; the counting kernels skip their work once the flag
// is set.
__device__ inline int uf_find(int* parent, int a, int limit, long long* gave_up) {
    int p = ((volatile int*)parent)[a];
    for (int it = 0; p != a; ++it) {
        if (it >= limit) {
            *(volatile long long*)gave_up = 1;
            break;
        }
        const int gp = ((volatile int*)parent)[p];
        if (gp != p) atomicCAS(&parent[a], p, gp);   // path halving
        a = p;
        p = gp;
    }
    return a;
}

__device__ inline void uf_union(int* parent, int a, int b, int limit, long long* gave_up) {
    for (int it = 0; it < limit; ++it) {
        a = uf_find(parent, a, limit, gave_up);
        b = uf_find(parent, b, limit, gave_up);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(&parent[a], a, b) == a) return;
    }
    *(volatile long long*)gave_up = 1;
}

constexpr int kCW = 4;   // warps per block

__device__ __forceinline__ float ex2f_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
constexpr float kBand = 1e-3f;   // fm^2, far above the FP32 screening error

struct Frame {
    float Lhi, Llo, iL;
    int wrap;
};

__device__ inline Frame frame_of(const SysState* st) {
    Frame f;
    f.Lhi = (float)st->L;
    f.Llo = (float)(st->L - (double)f.Lhi);
    f.iL = (float)(1.0 / st->L);
    f.wrap = st->need_wrap;
    return f;
}

// Source data of tile J for this lane, loaded ahead of its use (the loads of
// the next list entry are in flight while the current one is evaluated).
struct SrcLoad {
    float4 h, l, oJ;
};

__device__ __forceinline__ SrcLoad load_src(const SysConst& S, int J, int lane) {
    SrcLoad r;
    r.h = S.xhi[J * kTile + lane];
    r.l = S.xlo[J * kTile + lane];
    r.oJ = *reinterpret_cast<const float4*>(&S.torgf[4 * J]);
    return r;
}

// The loaded source moved to the image next to tile I (origin oI): an
// error-free two-sum on the hi + lo pair.
__device__ inline void shift_src(const SrcLoad& r, const float4& oI, const Frame& F, float4& h, float4& l) {
    h = r.h;
    l = r.l;
    const float s[3] = {rintf((oI.x - r.oJ.x) * F.iL), rintf((oI.y - r.oJ.y) * F.iL), rintf((oI.z - r.oJ.z) * F.iL)};
    float* hp = &h.x;
    float* lp = &l.x;
    for (int a = 0; a < 3; ++a) {
        if (s[a] != 0.0f) {
            const float b = s[a] * F.Lhi;
            const float t = hp[a] + b;
            const float bb = t - hp[a];
            const float e = (hp[a] - (t - bb)) + (b - bb);
            hp[a] = t;
            lp[a] = lp[a] + s[a] * F.Llo + e;
        }
    }
}

// Bounding box of the warp's valid targets (FP32 high parts) and the test
// of a source against it: a source farther than the reach from the box has
// no pair inside the cutoff with any target, so it is not queued.  The high
// parts are within 2^-24 |x| (< 1e-4 fm below 1000 fm) of the positions,
// far inside the reach margin kReachMargin.
struct WBox {
    float cx, cy, cz, hx, hy, hz;
};
constexpr float kReachMargin = 0.01f;   // fm

__device__ inline WBox warp_box(const float4& hi, bool valid) {
    float mn[3] = {valid ? hi.x : INFINITY, valid ? hi.y : INFINITY, valid ? hi.z : INFINITY};
    float mx[3] = {valid ? hi.x : -INFINITY, valid ? hi.y : -INFINITY, valid ? hi.z : -INFINITY};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
    WBox b;
    b.cx = 0.5f * (mn[0] + mx[0]);
    b.cy = 0.5f * (mn[1] + mx[1]);
    b.cz = 0.5f * (mn[2] + mx[2]);
    b.hx = 0.5f * (mx[0] - mn[0]);
    b.hy = 0.5f * (mx[1] - mn[1]);
    b.hz = 0.5f * (mx[2] - mn[2]);
    return b;
}

__device__ __forceinline__ bool near_box(const WBox& b, const float4& q, float reach2) {
    const float gx = fmaxf(fabsf(q.x - b.cx) - b.hx, 0.0f);
    const float gy = fmaxf(fabsf(q.y - b.cy) - b.hy, 0.0f);
    const float gz = fmaxf(fabsf(q.z - b.cz) - b.hz, 0.0f);
    return fmaf(gz, gz, fmaf(gy, gy, gx * gx)) < reach2;
}

__device__ inline float d2_screen(const float4& hi, const float4& lo, const float4& q, const float4& u,
                                  const Frame& F) {
    float dx = (hi.x - q.x) + (lo.x - u.x);
    float dy = (hi.y - q.y) + (lo.y - u.y);
    float dz = (hi.z - q.z) + (lo.z - u.z);
    if (F.wrap) {
        const float kx = rintf(dx * F.iL), ky = rintf(dy * F.iL), kz = rintf(dz * F.iL);
        dx = fmaf(-F.Llo, kx, fmaf(-F.Lhi, kx, dx));
        dy = fmaf(-F.Llo, ky, fmaf(-F.Lhi, ky, dy));
        dz = fmaf(-F.Llo, kz, fmaf(-F.Lhi, kz, dz));
    }
    return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

}  // namespace

// Proton slots [0, Np): parent = self; minid/zc/ac cleared; outputs cleared.
__global__ void k_cl_init(EngineDev E, int only) {
    const SysConst& S = E.sys[only];
    const ClusterBufs& B = *S.cl;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < S.Np) {
        B.parent[i] = i;
        B.minid[i] = 0x7fffffff;
        B.zc[i] = 0;
        B.ac[i] = 0;
    }
    if (i <= S.N) B.hist_A[i] = 0;
    if (i <= S.Np) B.hist_Z[i] = 0;
    if (i < 8) B.stats[i] = 0;
}

// Warp per proton tile: proton pairs closer than r_pp.  Each unordered pair
// is found once, from the tile of its smaller slot (source tiles J < I hold
// no such pair and are skipped; the lists are in increasing J).  The pairs
// found collect in a per-warp shared buffer that is appended to the edge
// buffer with one atomic per flush, and k_cl_union unites them, one thread
// per edge; a pair beyond the edge buffer's capacity is united here.
constexpr int kEB = 96;   // per-warp shared edge buffer (a flush leaves room for a full warp)

__device__ __forceinline__ void flush_edges(const ClusterBufs& B, const SysConst& S, int2* buf, int& ne, int lane) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(reinterpret_cast<unsigned long long*>(&B.stats[6]), (unsigned long long)ne);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int i = lane; i < ne; i += 32) {
        const int2 ed = buf[i];
        if (base + i < (unsigned long long)B.ecap) B.edges[base + i] = ed;
        else uf_union(B.parent, ed.x, ed.y, S.uf_limit, &B.stats[7]);
    }
    __syncwarp();
    ne = 0;
}

__global__ void k_cl_link(EngineDev E, int only) {
    __shared__ float4 sh[kCW][kTile], sl[kCW][kTile];
    __shared__ int sq[kCW][kTile];
    __shared__ int2 sedge[kCW][kEB];
    const SysConst& S = E.sys[only];
    const ClusterBufs& B = *S.cl;
    const int I = blockIdx.x * kCW + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (I >= S.Tp) return;
    const SysState* st = S.st;
    const Frame F = frame_of(st);
    const double L = st->L, hL = 0.5 * L, r2c = S.r_pp * S.r_pp;
    const float lo2 = (float)r2c - kBand, hi2 = (float)r2c + kBand;
    const int N = S.N;
    const double* x = S.x[st->cur];
    const int p = I * kTile + lane;
    const bool valid = p < S.Np;
    const float4 hi = S.xhi[I * kTile + lane], lo = S.xlo[I * kTile + lane];
    const float4 oI = *reinterpret_cast<const float4*>(&S.torgf[4 * I]);
    const WBox box = warp_box(hi, valid);
    const float reach = sqrtf(hi2) + kReachMargin, reach2 = reach * reach;
    int2* buf = sedge[w];
    int ne = 0;
    const int e1 = B.start[I + 1];
    int e = B.start[I];
    while (e < e1 && B.list[e] < I) ++e;
    int Jn = e < e1 ? B.list[e] : 0;
    SrcLoad nx;
    if (e < e1) nx = load_src(S, Jn, lane);
    while (e < e1) {
        const int J = Jn;
        const SrcLoad cur = nx;
        if (++e < e1) {
            Jn = B.list[e];
            nx = load_src(S, Jn, lane);
        }
        float4 h, l;
        shift_src(cur, oI, F, h, l);
        const int q = J * kTile + lane;
        const bool pass = q < S.Np && (F.wrap || near_box(box, h, reach2));
        const unsigned mp = __ballot_sync(0xffffffffu, pass);
        if (!mp) continue;
        __syncwarp();
        if (pass) {
            const int at = __popc(mp & ((1u << lane) - 1u));
            sh[w][at] = h;
            sl[w][at] = l;
            sq[w][at] = q;
        }
        __syncwarp();
        const int nq = __popc(mp);
        for (int k = 0; k < nq; ++k) {
            const int qq = sq[w][k];
            bool link = false;
            if (valid && qq > p) {
                const float d2 = d2_screen(hi, lo, sh[w][k], sl[w][k], F);
                link = d2 < lo2;
                if (!link && d2 < hi2)
                    link = d2_exact(x[p], x[N + p], x[2 * N + p], x[qq], x[N + qq], x[2 * N + qq], L, hL) < r2c;
            }
            const unsigned m = __ballot_sync(0xffffffffu, link);
            if (!m) continue;
            if (ne + 32 > kEB) flush_edges(B, S, buf, ne, lane);
            if (link) buf[ne + __popc(m & ((1u << lane) - 1u))] = make_int2(p, qq);
            __syncwarp();
            ne += __popc(m);
        }
    }
    if (ne) flush_edges(B, S, buf, ne, lane);
}

// One thread per buffered link: unite its two protons.
__global__ void k_cl_union(EngineDev E, int only) {
    const SysConst& S = E.sys[only];
    const ClusterBufs& B = *S.cl;
    const long long n = min((long long)B.stats[6], B.ecap);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int2 ed = B.edges[i];
        uf_union(B.parent, ed.x, ed.y, S.uf_limit, &B.stats[7]);
    }
}

// Smallest original index per component (and each proton pointed at its
// root).  Lanes of a warp with the same root combine first (one atomic per
// root and warp: a large cluster would otherwise serialise every proton's
// atomic on one address).
__global__ void k_cl_minid(EngineDev E, int only) {
    const SysConst& S = E.sys[only];
    const ClusterBufs& B = *S.cl;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = q < S.Np;
    const int r = ok ? uf_find(B.parent, q, S.uf_limit, &B.stats[7]) : -1 - (int)(threadIdx.x & 31);
    // the links are all united: point q at its root, so later finds take one step
    if (ok && r != q) B.parent[q] = r;
    int id = ok ? S.id[S.st->cur][q] : 0x7fffffff;
    const unsigned same = __match_any_sync(0xffffffffu, r);
    const int lane = threadIdx.x & 31;
    for (unsigned m = same; m; m &= m - 1) id = min(id, __shfl_sync(same, id, __ffs(m) - 1));
    if (ok && lane == __ffs(same) - 1) atomicMin(&B.minid[r], id);
}

// Proton labels; neutron assignment (warp per neutron tile).
__global__ void k_cl_assign(EngineDev E, int only) {
    __shared__ float4 sh[kCW][kTile], sl[kCW][kTile];
    __shared__ int sid[kCW][kTile], sq[kCW][kTile];
    const SysConst& S = E.sys[only];
    const ClusterBufs& B = *S.cl;
    const int I = blockIdx.x * kCW + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (I >= S.T) return;
    const SysState* st = S.st;
    const int c = st->cur, N = S.N;
    const double* x = S.x[c];
    const int p = tile_slot0(S, I) + lane;
    const bool valid = p < tile_end(S, I);
    if (I < S.Tp) {
        if (valid) B.label[p] = B.minid[uf_find(B.parent, p, S.uf_limit, &B.stats[7])];
        return;
    }
    const Frame F = frame_of(st);
    const double L = st->L, hL = 0.5 * L, r2c = S.r_np * S.r_np;
    const float hi2 = (float)r2c + kBand;
    const float4 hi = S.xhi[I * kTile + lane], lo = S.xlo[I * kTile + lane];
    const float4 oI = *reinterpret_cast<const float4*>(&S.torgf[4 * I]);
    const double xi = valid ? x[p] : 0, yi = valid ? x[N + p] : 0, zi = valid ? x[2 * N + p] : 0;
    const WBox box = warp_box(hi, valid);
    const float reach = sqrtf(hi2) + kReachMargin, reach2 = reach * reach;
    // The nearest candidate by the exact rule (FP64 squared distance, then the
    // smaller original index), with the FP64 distance evaluated only where the
    // FP32 screen cannot decide: the screened value is within a few ulp of
    // the FP64 one, far inside kBand, so a candidate more than kBand below
    // (above) the best is nearer (farther) in FP64 as well.  The best is the
    // exact minimum of the candidates; if it lies beyond r_np, so do all.
    float best_f = 0.0f;
    double best_d2 = 0.0;
    bool best_exact = false;
    int best_id = -1, best_slot = -1;
    for (int e = B.start[I]; e < B.start[I + 1]; ++e) {
        const int J = B.list[e];
        float4 h, l;
        shift_src(load_src(S, J, lane), oI, F, h, l);
        const int q = J * kTile + lane;
        const bool pass = q < S.Np && (F.wrap || near_box(box, h, reach2));
        const unsigned mp = __ballot_sync(0xffffffffu, pass);
        if (!mp) continue;
        __syncwarp();
        if (pass) {
            const int at = __popc(mp & ((1u << lane) - 1u));
            sh[w][at] = h;
            sl[w][at] = l;
            sid[w][at] = S.id[c][q];
            sq[w][at] = q;
        }
        __syncwarp();
        if (!valid) continue;
        const int nq = __popc(mp);
        for (int k = 0; k < nq; ++k) {
            const float d2f = d2_screen(hi, lo, sh[w][k], sl[w][k], F);
            if (d2f >= hi2) continue;
            const int qq = sq[w][k];
            const int oid = sid[w][k];
            if (best_slot < 0 || d2f < best_f - kBand) {
                best_f = d2f;
                best_exact = false;
                best_id = oid;
                best_slot = qq;
            } else if (d2f <= best_f + kBand) {
                const double d2 = d2_exact(xi, yi, zi, x[qq], x[N + qq], x[2 * N + qq], L, hL);
                if (!best_exact) {
                    best_d2 = d2_exact(xi, yi, zi, x[best_slot], x[N + best_slot], x[2 * N + best_slot], L, hL);
                    best_exact = true;
                }
                if (d2 < best_d2 || (d2 == best_d2 && oid < best_id)) {
                    best_f = d2f;
                    best_d2 = d2;
                    best_id = oid;
                    best_slot = qq;
                }
            }
        }
    }
    if (best_slot >= 0 && best_f >= (float)r2c - kBand) {
        if (!best_exact) best_d2 = d2_exact(xi, yi, zi, x[best_slot], x[N + best_slot], x[2 * N + best_slot], L, hL);
        if (!(best_d2 < r2c)) best_slot = -1;
    }
    if (valid) B.label[p] = best_slot < 0 ? -1 : B.minid[uf_find(B.parent, best_slot, S.uf_limit, &B.stats[7])];
}

// Per-cluster counts (labels are original proton indices < Np).  Lanes of a
// warp with the same label (and kind) add their counts in one atomic.
__global__ void k_cl_count(EngineDev E, int only) {
    const SysConst& S = E.sys[only];
    const ClusterBufs& B = *S.cl;
    if (B.stats[7]) return;      // a union-find loop gave up: labels are not valid
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool ok = p < S.N;
    const int lab = ok ? B.label[p] : -2;
    const bool prot = ok && p < S.Np;
    const unsigned same = __match_any_sync(0xffffffffu, lab);
    const unsigned nprot = __popc(same & __ballot_sync(0xffffffffu, prot));
    if (!ok || lane != __ffs(same) - 1) return;
    if (lab < 0) {
        atomicAdd((unsigned long long*)&B.stats[1], (unsigned long long)__popc(same));
        return;
    }
    atomicAdd(&B.ac[lab], __popc(same));
    if (nprot) atomicAdd(&B.zc[lab], (int)nprot);
}

// Histograms over clusters; labels written in original order.
__global__ void k_cl_hist(EngineDev E, int only, int32_t* labels_out) {
    const SysConst& S = E.sys[only];
    const ClusterBufs& B = *S.cl;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= S.N || B.stats[7]) return;   // (union-find gave up: labels are not valid)
    const int i = S.id[S.st->cur][p];
    const int lab = B.label[p];
    if (labels_out) labels_out[i] = lab;
    if (p < S.Np && lab == i) {
        const int A = B.ac[i], Z = B.zc[i];
        atomicAdd((unsigned long long*)&B.hist_A[A], 1ull);
        atomicAdd((unsigned long long*)&B.hist_Z[Z], 1ull);
        atomicAdd((unsigned long long*)&B.stats[0], 1ull);
        if (A >= 12) {
            atomicAdd((unsigned long long*)&B.stats[2], 1ull);
            atomicAdd((unsigned long long*)&B.stats[3], (unsigned long long)A);
            atomicAdd((unsigned long long*)&B.stats[4], (unsigned long long)Z);
        }
    }
}

// ------------------------------------------------------------------ MSTE
// Energy-criterion clusters, the minimum spanning tree in two-particle
// energy space that Sec. II.C names beside its distance algorithm (reading
// of the definition): nucleons i, j are bound when
//   e_ij = V_ij(r_ij) + (M/4) |v_i - v_j|^2 < 0,
// V_ij of Eq. (1) at the nearest image (nuclear part inside r_nuc; screened
// Coulomb for proton pairs, inside r_C when coulomb == 1, always when
// coulomb == 2).  Clusters are the connected components of bound pairs.
// Candidate pairs: the tile with itself and the near entries of the force
// lists (every pair inside r_nuc; pairs beyond have V >= 0).  Each pair is
// screened in FP32 (exact hi + lo separations, velocities rounded to FP32);
// pairs within a margin of the threshold take the decision of FP64
// arithmetic in a fixed order (no contraction):
//   r2 as for the distance clusters; g = exp(-r2 / (2 Lambda));
//   V = ((a g) g + s g) + [pp] (alpha exp(-sqrt(r2) / lambda)) / sqrt(r2);
//   e = V + (M/4) ((dvx dvx + dvy dvy) + dvz dvz).

namespace {

__device__ inline bool ms_bound_exact(const SysConst& S, const double* x, const double* v, int p, int q,
                                      double L, double hL) {
    const int N = S.N;
    const double r2 = d2_exact(x[p], x[N + p], x[2 * N + p], x[q], x[N + q], x[2 * N + q], L, hL);
    if (!(r2 < __dmul_rn(S.r_nuc, S.r_nuc))) return false;
    const bool pi = p < S.Np, pj = q < S.Np;
    const double sc = (pi == pj) ? __dadd_rn(S.b, S.c) : __dsub_rn(S.b, S.c);
    const double g = exp(__ddiv_rn(-r2, __dmul_rn(2.0, S.Lambda)));
    double V = __dadd_rn(__dmul_rn(__dmul_rn(S.a, g), g), __dmul_rn(sc, g));
    if (pi && pj && S.coulomb != 0 && (S.coulomb == 2 || r2 < __dmul_rn(S.r_C, S.r_C))) {
        const double r = __dsqrt_rn(r2);
        V = __dadd_rn(V, __ddiv_rn(__dmul_rn(S.alpha, exp(__ddiv_rn(-r, S.lambda_s))), r));
    }
    const double dx = __dsub_rn(v[p], v[q]), dy = __dsub_rn(v[N + p], v[N + q]), dz = __dsub_rn(v[2 * N + p], v[2 * N + q]);
    const double k = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return __dadd_rn(V, __dmul_rn(__dmul_rn(0.25, S.M), k)) < 0.0;
}

constexpr float kMsRel = 1e-4f;     // FP32 screening margin, relative to the terms' magnitudes
constexpr float kMsAbs = 1e-9f;     // and absolute (MeV)

}  // namespace

// All N slots: parent = self; minid, per-root counts, outputs cleared.
__global__ void k_ms_init(EngineDev E, int only) {
    const SysConst& S = E.sys[only];
    const ClusterBufs& B = *S.cl;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < S.N) {
        B.parent[i] = i;
        B.minid[i] = 0x7fffffff;
        B.zc[i] = 0;
        B.ac[i] = 0;
    }
    if (i <= S.N) B.hist_A[i] = 0;
    if (i <= S.Np) B.hist_Z[i] = 0;
    if (i < 8) B.stats[i] = 0;
}

// Warp per tile: every bound pair (i in I, j in I or a near entry).  Each
// source is queued only when it lies within the nuclear range of the box of
// the warp's targets (pairs beyond it are not bound: V >= 0 there); the bound
// pairs go to the edge buffer (united afterwards by k_cl_union, one thread
// per edge; beyond its capacity they are united here).
// half: the force lists hold each tile pair once and leave the tile itself
// out (split precision, tile lists); otherwise they are full.
__global__ void k_ms_link(EngineDev E, int only, int prec) {
    __shared__ float4 sh[kCW][kTile], sl[kCW][kTile], sv[kCW][kTile];
    __shared__ int sq[kCW][kTile];
    __shared__ int2 sedge[kCW][kEB];
    const SysConst& S = E.sys[only];
    const ClusterBufs& B = *S.cl;
    const int I = blockIdx.x * kCW + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (I >= S.T) return;
    const SysState* st = S.st;
    const Frame F = frame_of(st);
    const double L = st->L, hL = 0.5 * L;
    const int N = S.N, c = st->cur;
    const double* x = S.x[c];
    const double* v = S.v[c];
    const bool half = prec == 0 && S.list_kind == 0;
    const PairF& P = S.pf;
    const float far2 = P.rn2 + kBand, near2 = P.rn2 - kBand;
    const float a = (float)S.a, qM = (float)(0.25 * S.M);
    const int p0 = tile_slot0(S, I), p = p0 + lane;
    const bool valid = p < tile_end(S, I);
    const bool Ip = I < S.Tp;
    const float4 hi = S.xhi[I * kTile + lane], lo = S.xlo[I * kTile + lane];
    const float vx = valid ? (float)v[p] : 0.f, vy = valid ? (float)v[N + p] : 0.f, vz = valid ? (float)v[2 * N + p] : 0.f;
    const WBox box = warp_box(hi, valid);
    const float reach = sqrtf(far2) + kReachMargin, reach2 = reach * reach;
    int2* buf = sedge[w];
    int ne = 0;
    const int* lst = S.list + (long long)I * S.T;
    const int nnear = S.lnear[I];
    // source 0 .. nnear (+1 for the tile itself when the lists leave it out)
    const int nsrc = nnear + (half ? 1 : 0);
    for (int e = 0; e < nsrc; ++e) {
        int J = I, shk = kShiftNone;
        if (!half || e > 0) {
            const int ent = lst[half ? e - 1 : e];
            J = ent & kJMask;
            shk = (ent >> kShiftPos) & 63;
        }
        float4 h = S.xhi[J * kTile + lane], l = S.xlo[J * kTile + lane];
        if (shk != kShiftNone) apply_shift(shk, F.Lhi, F.Llo, h, l);
        const int q0 = tile_slot0(S, J), nJ = tile_end(S, J) - q0;
        const int qs = q0 + lane;
        const bool pass = lane < nJ && (F.wrap || near_box(box, h, reach2));
        const unsigned mp = __ballot_sync(0xffffffffu, pass);
        if (!mp) continue;
        __syncwarp();
        if (pass) {
            const int at = __popc(mp & ((1u << lane) - 1u));
            sh[w][at] = h;
            sl[w][at] = l;
            sv[w][at] = make_float4((float)v[qs], (float)v[N + qs], (float)v[2 * N + qs], 0.f);
            sq[w][at] = qs;
        }
        __syncwarp();
        const bool Jp = J < S.Tp;
        const bool pp = Ip && Jp;
        const bool coul = pp && S.coulomb != 0;
        const float sfac = (Ip == Jp) ? (float)(S.b + S.c) : (float)(S.b - S.c);
        const int nq = __popc(mp);
        for (int k = 0; k < nq; ++k) {
            const int q = sq[w][k];
            bool bound = false;
            // each pair of the tile with itself once
            if (valid && (J != I || q > p)) {
                const float r2 = d2_screen(hi, lo, sh[w][k], sl[w][k], F);
                if (r2 < far2) {
                    const float g = ex2f_approx(r2 * P.kq);
                    float V = g * fmaf(a, g, sfac);
                    float mag = g * fmaf(a, g, fabsf(sfac));
                    if (coul && (S.coulomb == 2 || r2 < P.rc2)) {
                        const float ri = rsqrtf(r2);
                        const float vc = ex2f_approx(fmaf(r2 * ri, P.kc, P.l2a)) * ri;
                        V += vc;
                        mag += vc;
                    }
                    const float4 u = sv[w][k];
                    const float dx = vx - u.x, dy = vy - u.y, dz = vz - u.z;
                    const float ke = qM * fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                    const float en = V + ke, band = kMsRel * (mag + ke) + kMsAbs;
                    // (a Coulomb cutoff inside the nuclear range: its edge is decided in FP64)
                    const bool cedge = coul && S.coulomb == 1 && fabsf(r2 - P.rc2) < kBand;
                    if (cedge) bound = ms_bound_exact(S, x, v, p, q, L, hL);
                    else if (en > band) bound = false;
                    else if (en < -band && r2 < near2) bound = true;
                    else bound = ms_bound_exact(S, x, v, p, q, L, hL);
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, bound);
            if (!m) continue;
            if (ne + 32 > kEB) flush_edges(B, S, buf, ne, lane);
            if (bound) buf[ne + __popc(m & ((1u << lane) - 1u))] = make_int2(p, q);
            __syncwarp();
            ne += __popc(m);
        }
    }
    if (ne) flush_edges(B, S, buf, ne, lane);
}

// Per root: smallest original index and component size.
__global__ void k_ms_root(EngineDev E, int only) {
    const SysConst& S = E.sys[only];
    const ClusterBufs& B = *S.cl;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= S.N) return;
    const int r = uf_find(B.parent, q, S.uf_limit, &B.stats[7]);
    atomicMin(&B.minid[r], S.id[S.st->cur][q]);
    atomicAdd(&B.ac[r], 1);
}

// Labels (a neutron alone in its component is free); counts cleared for
// the per-label pass.
__global__ void k_ms_label(EngineDev E, int only) {
    const SysConst& S = E.sys[only];
    const ClusterBufs& B = *S.cl;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= S.N) return;
    const int r = uf_find(B.parent, q, S.uf_limit, &B.stats[7]);
    B.label[q] = (q >= S.Np && B.ac[r] == 1) ? -1 : B.minid[r];
}

__global__ void k_ms_clear(EngineDev E, int only) {
    const SysConst& S = E.sys[only];
    const ClusterBufs& B = *S.cl;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= S.N) return;
    B.ac[q] = 0;
    B.zc[q] = 0;
}

// Histograms over clusters (the representative is the member whose original
// index is the label, of either species); labels written in original order.
__global__ void k_ms_hist(EngineDev E, int only, int32_t* labels_out) {
    const SysConst& S = E.sys[only];
    const ClusterBufs& B = *S.cl;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= S.N || B.stats[7]) return;   // (union-find gave up: labels are not valid)
    const int i = S.id[S.st->cur][p];
    const int lab = B.label[p];
    if (labels_out) labels_out[i] = lab;
    if (lab >= 0 && lab == i) {
        const int A = B.ac[i], Z = B.zc[i];
        atomicAdd((unsigned long long*)&B.hist_A[A], 1ull);
        atomicAdd((unsigned long long*)&B.hist_Z[Z], 1ull);
        atomicAdd((unsigned long long*)&B.stats[0], 1ull);
        if (A >= 12) {
            atomicAdd((unsigned long long*)&B.stats[2], 1ull);
            atomicAdd((unsigned long long*)&B.stats[3], (unsigned long long)A);
            atomicAdd((unsigned long long*)&B.stats[4], (unsigned long long)Z);
        }
    }
}

void launch_mste(const EngineHost& H, cudaStream_t s, int only, int N, int T, int32_t* d_labels_out) {
    const EngineDev& E = H.dev;
    const int n1 = (N + 1 + 255) / 256, n = (N + 255) / 256;
    H.rec("ms_init", s);
    k_ms_init<<<n1, 256, 0, s>>>(E, only);
    H.rec("ms_link", s);
    k_ms_link<<<(T + kCW - 1) / kCW, kCW * 32, 0, s>>>(E, only, H.precision);
    k_cl_union<<<std::min((N + 255) / 256, 148 * 16), 256, 0, s>>>(E, only);
    H.rec("ms_label", s);
    k_ms_root<<<n, 256, 0, s>>>(E, only);
    k_ms_label<<<n, 256, 0, s>>>(E, only);
    k_ms_clear<<<n, 256, 0, s>>>(E, only);
    k_cl_count<<<n, 256, 0, s>>>(E, only);
    H.rec("ms_hist", s);
    k_ms_hist<<<n, 256, 0, s>>>(E, only, d_labels_out);
    H.count(8);
}

void launch_clusters(const EngineHost& H, cudaStream_t s, int only, int Np, int N, int Tp, int T,
                     int32_t* d_labels_out) {
    const EngineDev& E = H.dev;
    const int n1 = (N + 1 + 255) / 256;
    H.rec("cl_init", s);
    k_cl_init<<<n1, 256, 0, s>>>(E, only);
    H.rec("cl_link", s);
    if (Tp > 0) {
        k_cl_link<<<(Tp + kCW - 1) / kCW, kCW * 32, 0, s>>>(E, only);
        k_cl_union<<<std::min((Np + 255) / 256, 148 * 16), 256, 0, s>>>(E, only);
    }
    H.rec("cl_minid", s);
    if (Np > 0) k_cl_minid<<<(Np + 255) / 256, 256, 0, s>>>(E, only);
    H.rec("cl_assign", s);
    k_cl_assign<<<(T + kCW - 1) / kCW, kCW * 32, 0, s>>>(E, only);
    H.rec("cl_count", s);
    k_cl_count<<<(N + 255) / 256, 256, 0, s>>>(E, only);
    H.rec("cl_hist", s);
    k_cl_hist<<<(N + 255) / 256, 256, 0, s>>>(E, only, d_labels_out);
    H.count(Tp > 0 ? 7 : 4);
}

}  // namespace pasta
