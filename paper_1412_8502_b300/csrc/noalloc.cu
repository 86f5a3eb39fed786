// md_clusters_noalloc: the cluster analysis for callers that cannot allocate
// device memory.
//
// Some callers hold their positions in device memory they manage themselves
// and may not call cudaMalloc at all: code that runs inside another
// application's memory pool or arena (where a foreign allocation breaks the
// host's accounting or fragments its pool), or real-time loops that must not
// stall on the allocator (cudaMalloc can wait on the device).  For them
// this entry point runs the same distance-linkage analysis as md_clusters on
// caller-provided device buffers, and all its working memory is one
// file-scope __device__ array of fixed size that every GPU loading the library
// keeps until the process exits.
//
// Limits and rules of use:
//  - at most kMaxN = 32768 nucleons; larger inputs are rejected with
//    MD_EINVAL before anything is launched;
//  - host code cannot use the array's symbol as a device address: each call
//    that is not being captured into a CUDA graph looks the address up with
//    cudaGetSymbolAddress in the context current at the call (a cached
//    address could belong to a context that was reset or to another context
//    on the same device); a call made while its stream is capturing uses the
//    address that the last uncaptured call on that device found, so make an
//    uncaptured call first, in the same context, before capturing one;
//  - the union-find loops are bounded (kNaLimit iterations, far above any
//    path an input within the size limit can produce); a loop that reaches
//    the bound sets d_counts[0] = -1 and the labels are then not valid;
//  - every call on a device shares the one array, and each call clears the
//    parts it needs first; calls whose work overlaps on the GPU (different
//    streams, or several host threads) race and must be serialised by the
//    caller;
//  - candidate pairs come from a scan over all proton tiles (O(N_p^2) FP64
//    distance tests), which is why the size is capped.
#include <cuda_runtime.h>

#include <mutex>

#include "engine.h"

namespace pasta {
namespace {

constexpr int kMaxN = 32768;
constexpr int kNaWarps = 4;
constexpr int kNaLimit = 1 << 26;   // iterations of a union-find loop before it gives up

// Four int arrays of kMaxN entries (union-find parents, smallest index per
// root, protons and nucleons per cluster label: 512 KB) and the flag of a
// union-find loop that gave up.
struct NoAllocScratch {
    int parent[kMaxN];
    int minid[kMaxN];
    int zc[kMaxN];
    int ac[kMaxN];
    int gave_up;
};
static __device__ __align__(256) NoAllocScratch g_na_scratch;

std::mutex g_na_mu;
NoAllocScratch* g_na_ptr[64] = {nullptr};

__device__ __forceinline__ double na_d2(const double* a, const double* b, double L, double hL) {
    double d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double v = __dsub_rn(a[k], b[k]);
        if (v > hL) v = __dsub_rn(v, L);
        else if (v < -hL) v = __dadd_rn(v, L);
        d[k] = v;
    }
    double s = __dmul_rn(d[0], d[0]);
    s = __dadd_rn(s, __dmul_rn(d[1], d[1]));
    s = __dadd_rn(s, __dmul_rn(d[2], d[2]));
    return s;
}

// Bounded union-find: a loop that reaches kNaLimit records it in *gave_up
// (a walk that gives up returns the valid slot it reached).
__device__ inline int na_find(int* parent, int a, int* gave_up) {
    int p = ((volatile int*)parent)[a];
    for (int it = 0; p != a; ++it) {
        if (it >= kNaLimit) {
            *(volatile int*)gave_up = 1;
            break;
        }
        const int gp = ((volatile int*)parent)[p];
        if (gp != p) atomicCAS(&parent[a], p, gp);
        a = p;
        p = gp;
    }
    return a;
}

__device__ inline void na_union(int* parent, int a, int b, int* gave_up) {
    for (int it = 0; it < kNaLimit; ++it) {
        a = na_find(parent, a, gave_up);
        b = na_find(parent, b, gave_up);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(&parent[a], a, b) == a) return;
    }
    *(volatile int*)gave_up = 1;
}

__global__ void k_na_init(NoAllocScratch* W, int N, int Np, long long* hA, long long* hZ, long long* counts) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < Np) {
        W->parent[i] = i;
        W->minid[i] = 0x7fffffff;
        W->zc[i] = 0;
        W->ac[i] = 0;
    }
    if (i <= N) hA[i] = 0;
    if (i <= Np) hZ[i] = 0;
    if (i < 5) counts[i] = 0;
    if (i == 0) W->gave_up = 0;
}

// Warp per 32-proton tile I, all tiles J >= I: link pairs closer than r_pp.
__global__ void k_na_link(NoAllocScratch* W, const double* x, int Np, double L, double r2c) {
    __shared__ double sb[kNaWarps][kTile][3];
    const int I = blockIdx.x * kNaWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int Tp = (Np + kTile - 1) / kTile;
    if (I >= Tp) return;
    const double hL = 0.5 * L;
    const int p = I * kTile + lane;
    const bool valid = p < Np;
    double xi[3] = {0.0, 0.0, 0.0};
    if (valid)
        for (int k = 0; k < 3; ++k) xi[k] = x[3 * p + k];
    for (int J = I; J < Tp; ++J) {
        const int q = J * kTile + lane;
        __syncwarp();
        for (int k = 0; k < 3; ++k) sb[w][lane][k] = q < Np ? x[3 * q + k] : 0.0;
        __syncwarp();
        if (!valid) continue;
        const int nq = min(kTile, Np - J * kTile);
        for (int k = 0; k < nq; ++k) {
            const int qq = J * kTile + k;
            if (qq <= p) continue;
            if (na_d2(xi, sb[w][k], L, hL) < r2c) na_union(W->parent, p, qq, &W->gave_up);
        }
    }
}

__global__ void k_na_minid(NoAllocScratch* W, int Np) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Np) return;
    atomicMin(&W->minid[na_find(W->parent, q, &W->gave_up)], q);
}

// Labels of protons; nearest proton closer than r_np for each neutron
// (equal distances: the smaller proton index).
__global__ void k_na_assign(NoAllocScratch* W, const double* x, int N, int Np, double L, double r2c,
                            int32_t* labels) {
    __shared__ double sb[kNaWarps][kTile][3];
    const int I = blockIdx.x * kNaWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int p = I * kTile + lane;
    if (I * kTile >= N) return;
    const bool valid = p < N;
    if (p < Np) {
        labels[p] = W->minid[na_find(W->parent, p, &W->gave_up)];
    }
    const bool neutron = valid && p >= Np;
    if (!__any_sync(0xffffffffu, neutron)) return;
    const double hL = 0.5 * L;
    double xi[3] = {0.0, 0.0, 0.0};
    if (neutron)
        for (int k = 0; k < 3; ++k) xi[k] = x[3 * p + k];
    const int Tp = (Np + kTile - 1) / kTile;
    double best_d2 = 0.0;
    int best = -1;
    for (int J = 0; J < Tp; ++J) {
        const int q = J * kTile + lane;
        __syncwarp();
        for (int k = 0; k < 3; ++k) sb[w][lane][k] = q < Np ? x[3 * q + k] : 0.0;
        __syncwarp();
        if (!neutron) continue;
        const int nq = min(kTile, Np - J * kTile);
        for (int k = 0; k < nq; ++k) {
            const double d2 = na_d2(xi, sb[w][k], L, hL);
            if (d2 < r2c && (best < 0 || d2 < best_d2)) {   // increasing index: ties keep the smaller
                best_d2 = d2;
                best = J * kTile + k;
            }
        }
    }
    if (neutron) labels[p] = best < 0 ? -1 : W->minid[na_find(W->parent, best, &W->gave_up)];
}

__global__ void k_na_count(NoAllocScratch* W, const int32_t* labels, int N, int Np, long long* counts) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N || W->gave_up) return;      // (labels are not valid then)
    const int lab = labels[p];
    if (lab < 0) {
        atomicAdd((unsigned long long*)&counts[1], 1ull);
        return;
    }
    atomicAdd(&W->ac[lab], 1);
    if (p < Np) atomicAdd(&W->zc[lab], 1);
}

__global__ void k_na_hist(NoAllocScratch* W, const int32_t* labels, int Np, long long* hA, long long* hZ,
                          long long* counts) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Np || W->gave_up || labels[i] != i) return;
    const int A = W->ac[i], Z = W->zc[i];
    atomicAdd((unsigned long long*)&hA[A], 1ull);
    atomicAdd((unsigned long long*)&hZ[Z], 1ull);
    atomicAdd((unsigned long long*)&counts[0], 1ull);
    if (A >= 12) {
        atomicAdd((unsigned long long*)&counts[2], 1ull);
        atomicAdd((unsigned long long*)&counts[3], (unsigned long long)A);
        atomicAdd((unsigned long long*)&counts[4], (unsigned long long)Z);
    }
}

// A union-find loop that gave up marks the result as not valid.
__global__ void k_na_status(const NoAllocScratch* W, long long* counts) {
    if (W->gave_up) counts[0] = -1;
}

// Device address of the scratch array in the current context.  A call that
// is not being captured looks it up (cudaGetSymbolAddress: no allocation)
// and remembers it for the device; a call under stream capture takes the
// remembered address, so that no lookup (which may load the module) runs
// inside a capture.
int scratch_address(cudaStream_t s, NoAllocScratch** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(MD_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return fail(MD_ENODEV, "device index out of range");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return fail(MD_ECUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_na_scratch);
        if (e != cudaSuccess)
            return fail(MD_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_na_ptr[dev] = static_cast<NoAllocScratch*>(ptr);
    } else if (!g_na_ptr[dev]) {
        return fail(MD_EINVAL, "md_clusters_noalloc: the first call on a device must not be captured");
    }
    *out = g_na_ptr[dev];
    return MD_OK;
}

}  // namespace
}  // namespace pasta

extern "C" int md_clusters_noalloc(const double* d_x, int64_t N, int64_t Np, double L, double r_pp, double r_np,
                                   int32_t* d_labels, int64_t* d_hist_A, int64_t* d_hist_Z, int64_t* d_counts,
                                   void* stream) {
    using namespace pasta;
    if (!d_x || !d_labels || !d_hist_A || !d_hist_Z || !d_counts)
        return fail(MD_EINVAL, "md_clusters_noalloc: null buffer");
    if (N < 1 || Np < 0 || Np > N) return fail(MD_EINVAL, "md_clusters_noalloc: need 1 <= N and 0 <= Np <= N");
    if (N > kMaxN)
        return fail(MD_EINVAL, "md_clusters_noalloc: N = " + std::to_string(N) + " exceeds the fixed scratch limit of " +
                                   std::to_string(kMaxN) + " nucleons");
    if (!(L > 0.0) || !(r_pp > 0.0) || !(r_np > 0.0)) return fail(MD_EINVAL, "md_clusters_noalloc: L, r_pp, r_np > 0");
    cudaStream_t s = (cudaStream_t)stream;
    NoAllocScratch* W = nullptr;
    int rc = scratch_address(s, &W);
    if (rc) return rc;
    const int n = (int)N, np = (int)Np;
    const int Tp = (np + kTile - 1) / kTile, T = (n + kTile - 1) / kTile;
    long long* hA = (long long*)d_hist_A;
    long long* hZ = (long long*)d_hist_Z;
    long long* cnt = (long long*)d_counts;
    k_na_init<<<(n + 1 + 255) / 256, 256, 0, s>>>(W, n, np, hA, hZ, cnt);
    if (Tp > 0) {
        k_na_link<<<(Tp + kNaWarps - 1) / kNaWarps, kNaWarps * 32, 0, s>>>(W, d_x, np, L, r_pp * r_pp);
        k_na_minid<<<(np + 255) / 256, 256, 0, s>>>(W, np);
    }
    k_na_assign<<<(T + kNaWarps - 1) / kNaWarps, kNaWarps * 32, 0, s>>>(W, d_x, n, np, L, r_np * r_np, d_labels);
    k_na_count<<<(n + 255) / 256, 256, 0, s>>>(W, d_labels, n, np, cnt);
    if (np > 0) k_na_hist<<<(np + 255) / 256, 256, 0, s>>>(W, d_labels, np, hA, hZ, cnt);
    k_na_status<<<1, 1, 0, s>>>(W, cnt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(MD_ECUDA, std::string("md_clusters_noalloc: ") + cudaGetErrorString(e));
    return MD_OK;
}
