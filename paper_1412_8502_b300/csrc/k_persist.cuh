// One velocity-Verlet step of every system of an engine in a single
// persistent launch (the batched ensemble: many independent systems of
// uneven size, the paper's Y_p x T sweep, Sec. III.B).
//
// The launch is cooperative (all blocks resident at once) with one block of
// 256 threads per slot the occupancy allows.  Its blocks run the phases of
// a step in order, each phase spread over them (the same device code as the
// separate kernels, each block playing the blocks of the separate launch in
// turn), with a grid-wide barrier between phases:
//   kick-drift | rebuild decision | [cell build: histogram, bin scan (two
//   passes), scatter, move, tiles | lists: super-tiles, tile-pair lists]
//   (only when some system rebuilds) | pair forces | closing kick with the
//   force conversion | finalisation (clock, box, thermostat, energies) |
//   thermostat / affine rescale.
// Force work items (the work list of (system, tile part) items of all
// systems) are taken from a device counter in item order, heavy proton items
// first, four at a time by each group of four warps.  Every barrier wait is
// bounded by %globaltimer: a wait that exceeds the host-set limit
// (md_params.wait_limit_ns) raises an error flag, after which every block
// leaves at its next barrier, and the host reports MD_ETIMEOUT.  The barrier
// counter is cleared by a memset node before each launch.
//
// Each system's arithmetic is that of the separate kernels, in the same
// order: a system gives bitwise the same trajectory here as alone.
#pragma once

#include <mutex>

namespace pasta {

constexpr int kPBlock = 256;     // threads per block of the persistent step kernel
constexpr int kPWarps = kPBlock / 32;
static_assert(kPBlock == kBlock, "the per-tile bodies play blocks of kBlock threads");
static_assert(kPBlock == kRed, "the per-system reductions (finalisation) use kRed threads");
static_assert(kPWarps % kForceWarps == 0, "whole groups of force warps per block");

namespace {

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Barrier of the nthreads threads (whole warps) that use hardware barrier id.
__device__ __forceinline__ void named_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Grid-wide barrier: every block's thread 0 arrives on the counter and waits
// (bounded) until all blocks have arrived this many times.  Returns false
// (in every thread of the block) when the wait gave up or another block did.
__device__ __forceinline__ bool grid_barrier(PersistCtl* ctl, unsigned& target, unsigned long long limit_ns,
                                             int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        target += gridDim.x;
        __threadfence();
        atomicAdd(&ctl->bar, 1u);
        const unsigned long long t0 = global_ns();
        int ok = 1;
        while (ld_acquire_u32(&ctl->bar) < target) {
            if (*(volatile int*)&ctl->error || global_ns() - t0 > limit_ns) {
                ok = 0;
                atomicOr(&ctl->error, 1);
                break;
            }
            __nanosleep(100);
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// The bin scan for 256-thread blocks: chunks of kScanChunk bins (as the
// 1024-thread kernels), 32 bins per thread; the chunk counts, then each chunk
// from the sum of the counts before it.  Exact integer prefix sums: the
// result does not depend on the chunking.
constexpr int kPScanPer = kScanChunk / kPBlock;
static_assert(kPScanPer % kScanPer == 0, "whole groups of 8 bins per thread");

__device__ __forceinline__ void pscan_reduce(const EngineDev& E, int vb) {
    __shared__ unsigned sm[33];
    const long long base = (long long)vb * kScanChunk + threadIdx.x * kPScanPer;
    unsigned s = 0;
#pragma unroll
    for (int q = 0; q < kPScanPer / kScanPer; ++q) {
        unsigned v[kScanPer];
        load8(E.hist, base + q * kScanPer, E.nbins_total, v);
        for (int k = 0; k < kScanPer; ++k) s += v[k];
    }
    unsigned tot;
    block_exscan(s, sm, &tot);
    if (threadIdx.x == 0) E.blocksum[vb] = tot;
}

__device__ __forceinline__ void pscan_bins(const EngineDev& E, int vb) {
    __shared__ unsigned sm[33];
    const unsigned off = chunk_offset(E, vb, sm);
    const long long base = (long long)vb * kScanChunk + threadIdx.x * kPScanPer;
    unsigned v[kPScanPer / kScanPer][kScanPer];
    unsigned s = 0;
#pragma unroll
    for (int q = 0; q < kPScanPer / kScanPer; ++q) {
        load8(E.hist, base + q * kScanPer, E.nbins_total, v[q]);
        for (int k = 0; k < kScanPer; ++k) s += v[q][k];
    }
    unsigned run = block_exscan(s, sm, nullptr) + off;
#pragma unroll
    for (int q = 0; q < kPScanPer / kScanPer; ++q) {
        unsigned o[kScanPer];
        for (int k = 0; k < kScanPer; ++k) {
            o[k] = run;
            run += v[q][k];
        }
        store8(E.binstart, base + q * kScanPer, E.nbins_total, o);
        store8(E.cursor, base + q * kScanPer, E.nbins_total, o);
    }
}

template <bool kEnergy, int kVar>
__global__ void __launch_bounds__(kPBlock, 2)
    k_step_persistent(EngineDev E, PersistCtl* ctl, unsigned long long limit_ns) {
    extern __shared__ float4 dyn_smem[];
    WarpQueues* fq = reinterpret_cast<WarpQueues*>(dyn_smem);   // force phase: one per warp
    __shared__ int s_ok;
    __shared__ int s_item[kPWarps / kForceWarps];
    unsigned target = 0;
    const int G = gridDim.x, b0 = blockIdx.x;
    const int nb = (E.ntiles + kTilesPerBlock - 1) / kTilesPerBlock;
#define PASTA_BARRIER() \
    if (!grid_barrier(ctl, target, limit_ns, &s_ok)) return

    for (int b = b0; b < nb; b += G) kick_drift_body<float>(E, b);
    PASTA_BARRIER();
    if (b0 == 0) {
        decide_body(E, 0, -1, 0, 0, 0, 0, 0);
        if (threadIdx.x == 0) ctl->work = 0;
    }
    PASTA_BARRIER();
    if (*(volatile int*)E.any_rebuild) {
        const int nscan = (int)((E.nbins_total + kScanChunk - 1) / kScanChunk);
        for (int b = b0; b < nb; b += G) hist_body(E, b);
        PASTA_BARRIER();
        for (int b = b0; b < nscan; b += G) pscan_reduce(E, b);
        PASTA_BARRIER();
        for (int b = b0; b < nscan; b += G) pscan_bins(E, b);
        PASTA_BARRIER();
        for (int b = b0; b < nb; b += G) scatter_body(E, b);
        PASTA_BARRIER();
        for (int b = b0; b < nb; b += G) move_body(E, b);
        PASTA_BARRIER();
        for (int b = b0; b < nb; b += G) tiles_body(E, b);
        PASTA_BARRIER();
        for (int b = b0; b < nb; b += G) super_body(E, b);
        PASTA_BARRIER();
        for (int b = b0; b < nb; b += G) lbuild_body(E, 1, b);
        PASTA_BARRIER();
    }
    {
        // Force work items from the device counter, four at a time per group
        // of four warps (half a block): the four items of a group are the same
        // part of four adjacent tiles, whose sources the warps then share in
        // L1, as the four warps of a block of the separate force kernel do.
        const int w = threadIdx.x >> 5, grp = threadIdx.x >> 7;
        for (;;) {
            if ((threadIdx.x & 127) == 0) s_item[grp] = (int)atomicAdd(&ctl->work, (unsigned)kForceWarps);
            named_sync(1 + grp, 128);
            const int g0 = s_item[grp];
            named_sync(1 + grp, 128);          // every warp of the group has read it
            if (g0 >= E.nitems) break;
            force_split_item<kEnergy, kVar>(E, -1, g0 + (w & (kForceWarps - 1)), fq[w]);
        }
    }
    PASTA_BARRIER();
    for (int b = b0; b < nb; b += G) kick_fix_body(E, b);
    PASTA_BARRIER();
    for (int s = b0; s < E.nsys; s += G) finalize_body(E, kEnergy ? 1 : 0, s);
    PASTA_BARRIER();
    rescale_body(E, -1, b0, G);
#undef PASTA_BARRIER
}

// Blocks per SM of each instantiation (0: not possible; -1: not yet set) per
// device, set by prepare_step_persistent outside any stream capture with the
// device current (function attributes belong to a device's context).
constexpr int kMaxDev = 64;
int g_persist_blocks[kMaxDev][2][3];
bool g_persist_init = false;

int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return -1;
    return dev;
}

template <bool kEnergy, int kVar>
int prepare_variant(int dev) {
    auto kern = k_step_persistent<kEnergy, kVar>;
    const size_t dsm = sizeof(WarpQueues) * kPWarps;
    int nb = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kPBlock, dsm) != cudaSuccess)
        return -1;
    g_persist_blocks[dev][kEnergy ? 1 : 0][kVar] = nb;
    return nb > 0 ? 0 : -1;
}

template <bool kEnergy, int kVar>
int step_persistent_variant(const EngineHost& H, cudaStream_t s, PersistCtl* ctl, unsigned long long limit_ns) {
    const int dev = current_device();
    if (dev < 0) return -1;
    const int bps = g_persist_blocks[dev][kEnergy ? 1 : 0][kVar];
    if (bps < 1) return -1;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(std::min(bps, 2) * sms));
    cfg.blockDim = dim3(kPBlock);
    cfg.dynamicSmemBytes = sizeof(WarpQueues) * kPWarps;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaMemsetAsync(&ctl->bar, 0, sizeof(unsigned), s) != cudaSuccess) return -1;
    if (cudaLaunchKernelEx(&cfg, k_step_persistent<kEnergy, kVar>, H.dev, ctl, limit_ns) != cudaSuccess) return -1;
    return 0;
}

}  // namespace

// Dynamic shared memory and occupancy of the persistent step kernel: call
// outside stream capture before its first launch; 0, or -1 if it cannot run
// (the CUDA error is left for the caller to read).  Done once per device, for
// the device current at the call.
int prepare_step_persistent() {
    static std::mutex mu;                // engines may be created from several host threads
    std::lock_guard<std::mutex> lk(mu);
    if (!g_persist_init) {
        for (auto& d : g_persist_blocks)
            for (auto& e : d)
                for (int& v : e) v = -1;
        g_persist_init = true;
    }
    const int dev = current_device();
    if (dev < 0) return -1;
    if (g_persist_blocks[dev][0][0] >= 0) return g_persist_blocks[dev][0][0] > 0 ? 0 : -1;
    int rc = prepare_variant<false, 0>(dev);
    if (!rc) rc = prepare_variant<false, 1>(dev);
    if (!rc) rc = prepare_variant<false, 2>(dev);
    if (!rc) rc = prepare_variant<true, 0>(dev);
    if (!rc) rc = prepare_variant<true, 1>(dev);
    if (!rc) rc = prepare_variant<true, 2>(dev);
    return rc;
}

// One step of every system in one cooperative launch (after a memset of the
// barrier counter).  var: force-pass code variant (0 long, 1 compact, 2
// minimal).  Returns 0, or -1 if the launch could not be made (the CUDA
// error is left for the caller to read).
int launch_step_persistent(const EngineHost& H, cudaStream_t s, bool energy, int var, PersistCtl* ctl,
                           unsigned long long limit_ns) {
    H.rec("step", s);
    int rc;
    if (energy) {
        rc = var == 0   ? step_persistent_variant<true, 0>(H, s, ctl, limit_ns)
             : var == 1 ? step_persistent_variant<true, 1>(H, s, ctl, limit_ns)
                        : step_persistent_variant<true, 2>(H, s, ctl, limit_ns);
    } else {
        rc = var == 0   ? step_persistent_variant<false, 0>(H, s, ctl, limit_ns)
             : var == 1 ? step_persistent_variant<false, 1>(H, s, ctl, limit_ns)
                        : step_persistent_variant<false, 2>(H, s, ctl, limit_ns);
    }
    H.count(1);
    return rc;
}

}  // namespace pasta
