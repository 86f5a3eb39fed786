// Launchers of the device kernels and the host view of an engine.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "md_device.cuh"

namespace pasta {

// Launch with programmatic stream serialization: the kernel may be scheduled
// before the kernel ahead of it on the stream has finished, and waits for it
// with griddep_wait() before touching any data (every kernel launched this
// way starts with that wait).  Used for the chains of short kernels of a step
// (kick-drift and decision; the cell and list builds; kick, finalisation and
// rescale): 4.5% off the cell build at 409,600 and 1% over the 51,200
// schedule.  The force kernels are launched plainly: with it the 51,200
// schedule was 1% slower.  Launch errors are left for cudaGetLastError.
template <typename... P, typename... A>
inline void launch_dep(void (*k)(P...), dim3 grid, dim3 block, cudaStream_t s, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    (void)cudaLaunchKernelEx(&cfg, k, static_cast<P>(args)...);
}

// Buffers of the on-demand cluster analysis (allocated on first use).
struct ClusterBufs {
    int* parent;             // [N] union-find over sorted slots (protons only for Sec. II.C)
    int* minid;              // [N] smallest original index per root
    int* zc;                 // [N] protons per cluster label
    int* ac;                 // [N] nucleons per cluster label (per root in the MSTE pass)
    int* label;              // [N] label per sorted slot
    long long* hist_A;       // [N+1]
    long long* hist_Z;       // [Np+1]
    long long* stats;        // [8]: clusters, free, big, sumA, sumZ; [6] links found; [7] a loop gave up
    int2* edges;             // [ecap] links (slot pairs) found by a link pass, united afterwards
    long long ecap;
    int* count;              // [T] candidate tiles per tile
    int* start;              // [T+1]
    int* list;               // [cap]
    long long cap;
    long long* total;        // [1] entries needed
};

// Host-side view passed to the launchers: device tables plus instrumentation
// (event records for per-kernel timing and a launch counter).
struct EngineHost {
    EngineDev dev;
    int precision = 0;
    bool any_pp = false;     // some system uses the all-pairs Coulomb (coulomb = 2)
    bool any_verlet = false; // some system uses per-particle Verlet lists (list_kind 1)
    int fixed_var = 0;       // force-pass variant of launches outside step graphs (system 0's force_unroll)
    void* owner = nullptr;   // Engine*, for rec/count callbacks
    void (*rec_fn)(void*, const char*, cudaStream_t) = nullptr;
    void (*count_fn)(void*, int) = nullptr;
    void rec(const char* name, cudaStream_t s) const {
        if (rec_fn) rec_fn(owner, name, s);
    }
    void count(int n) const {
        if (count_fn) count_fn(owner, n);
    }
};

void launch_rebuild(const EngineHost& H, cudaStream_t s, int forced_only, int only);
void launch_decide(const EngineHost& H, cudaStream_t s, int forced_only, int only,
                   cudaGraphConditionalHandle cond_cell, cudaGraphConditionalHandle cond_list, bool set_cond,
                   cudaGraphConditionalHandle cond_var, bool set_var);
void launch_cell_build(const EngineHost& H, cudaStream_t s, bool rec);
void launch_list_build(const EngineHost& H, cudaStream_t s, bool rec);
void launch_cluster_lists(const EngineHost& H, cudaStream_t s, int phase, int only);
void launch_force(const EngineHost& H, cudaStream_t s, bool energy, int only, int out_alt);
// The force pass in three parts, for step graphs: energy clear; the split
// kernel of one code variant (gate: the kernel returns at once unless the
// variant is this step's selection); the Verlet-list pass, the fixed-point
// conversion and the all-pairs Coulomb term.
// clear: launch the energy clear (step graphs leave it to k_decide); fix:
// launch k_force_fix (step graphs may fuse it into the closing kick).
void launch_force_pre(const EngineHost& H, cudaStream_t s, bool energy, int only, bool clear = true);
void launch_force_variant(const EngineHost& H, cudaStream_t s, bool energy, int only, int var, bool gate);
void launch_force_post(const EngineHost& H, cudaStream_t s, bool energy, int only, int out_alt, bool fix = true);
void launch_coulomb_pp(const EngineHost& H, cudaStream_t s, bool energy, int only, int out_alt);
void launch_init(const EngineHost& H, cudaStream_t s, const unsigned long long* d_seeds);
void launch_sd_update(const EngineHost& H, cudaStream_t s);
void launch_kick_drift(const EngineHost& H, cudaStream_t s);
// fused_fix: the closing kick also converts the split force pass's
// fixed-point accumulators (the force pass was launched without k_force_fix).
void launch_kick_finalize(const EngineHost& H, cudaStream_t s, bool energy, bool fused_fix);
void launch_energy_now(const EngineHost& H, cudaStream_t s, int only, double* d_out);
void launch_gather(const EngineHost& H, cudaStream_t s, int only, double* ox, double* ov, double* of,
                   int8_t* otype);
void launch_scatter_state(const EngineHost& H, cudaStream_t s, int only, const double* ix, const double* iv);
void launch_load_sorted(const EngineHost& H, cudaStream_t s, int only, const double* ix, const double* iv,
                        double L);
void launch_scatter_forces(const EngineHost& H, cudaStream_t s, int only, const double* iforce);
void launch_set_clock(const EngineHost& H, cudaStream_t s, int only, const double* d_clock,
                      bool keep_tiles = false);
void launch_set_rate(const EngineHost& H, cudaStream_t s, int only, double xi_dot);
// After a force re-evaluation outside a step: L_F = L.
void launch_mark_forces(const EngineHost& H, cudaStream_t s, int only);
void launch_clusters(const EngineHost& H, cudaStream_t s, int only, int Np, int N, int Tp, int T,
                     int32_t* d_labels_out);
void launch_mste(const EngineHost& H, cudaStream_t s, int only, int N, int T, int32_t* d_labels_out);
// One step of all systems as one persistent cooperative launch (after a
// memset node clearing the barrier counter); returns 0 or -1 (launch failed).
int launch_step_persistent(const EngineHost& H, cudaStream_t s, bool energy, int var, PersistCtl* ctl,
                           unsigned long long limit_ns);
int prepare_step_persistent();

}  // namespace pasta
