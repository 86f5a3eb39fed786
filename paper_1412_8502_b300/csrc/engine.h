// Host engine: owns the device memory of one or more systems, the global
// tables the multi-system kernels work over, the captured CUDA graphs of the
// step and relaxation loops, and per-kernel timing.
#pragma once
#include <cstddef>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "../../include/md.h"
#include "kernels.h"

namespace pasta {

struct SysHost {
    int64_t N = 0, Np = 0;
    int T = 0, Tp = 0, Tpad = 0;
    int nbits = 0;
    long long nbins = 0;
    double L0 = 0, rho = 0, Yp = 0, T0 = 0;
    uint64_t seed = 0;
    md_params prm{};
    SysConst c{};            // device pointers + constants (host copy)
    SysState* d_st = nullptr;
    ClusterBufs hcl{};       // host copy of the cluster buffer pointers
    ClusterBufs* d_cl = nullptr;
    bool cl_ready = false;
    double* d_stage = nullptr;   // [3N] x 3 staging (x, v, f) in original order
    int8_t* d_stage_t = nullptr;
    int32_t* d_stage_lab = nullptr;
    std::vector<void*> allocs;
    size_t bytes = 0;
    int64_t host_step = 0;   // steps since creation (mirror of the device count)
    double xi = 0.0;         // expansion rate in use
    bool dirty = false;      // forces must be re-evaluated before use
};

struct GraphRec {
    cudaGraphExec_t exec = nullptr;
    int nodes = 0;                      // kernels launched on every replay
    int cond_nodes = 0;                 // kernels of the conditional rebuild bodies
    std::vector<std::string> names;     // timing mode: one per event interval
    std::vector<cudaEvent_t> events;
};

class Engine {
public:
    // priority: of the engine's own stream (CUDA stream priority; 0 = default,
    // lower values are scheduled first where the device supports it)
    explicit Engine(int priority = 0);
    ~Engine();

    // Allocate and register a system; returns MD_OK or an error code.
    int add_system(int64_t N, double Yp, double rho, double T, uint64_t seed, const md_params& p);
    // Build the global tables after the set of systems changed.
    int build_tables();
    // Seed, relax and evaluate forces of all systems (creation path).
    int initialise();
    // Same, only enqueued on the engine's stream (no synchronisation).
    // relax = false leaves the relaxation iterations to relax_async.
    int initialise_async(bool relax = true);
    // Enqueue n steepest-descent relaxation iterations (serving: in slices).
    int relax_async(int64_t n);
    // Relaxation iterations the systems ask for (the largest relax_iters).
    int64_t relax_iters() const;
    // Release a system's device memory and drop it from the engine.
    void remove_system(int idx);

    int step(int64_t n, const std::vector<double>* xi_per_sys);
    // Enqueue n steps without synchronising (serving); events (n+1, may be
    // null) are recorded on the stream around every step.
    int step_async(int64_t n, const std::vector<double>* xi_per_sys, cudaEvent_t* events);
    // Device bytes a system with these arguments would allocate (engine of one).
    static size_t estimate_bytes(int64_t N, double Yp, double rho, const md_params& p);
    int refresh(int only);                  // forced rebuild + forces
    int forces(int idx, double* f_out);
    int energy(int idx, md_energy_t* e);
    int step_energy(int idx, md_energy_t* e);
    int clusters(int idx, int32_t* labels, int64_t* hA, int64_t* hZ, md_cluster_stats* st);
    int clusters_mste(int idx, int32_t* labels, int64_t* hA, int64_t* hZ, md_cluster_stats* st);
    int get_state(int idx, md_state_view* v);
    int set_state(int idx, const md_state_view* v);
    int set_params(int idx, const md_params& p);
    int info(int idx, md_info_t* out);
    int autotune(int64_t steps, md_params* chosen);
    int check_errors();                     // sync + MD_ENUMERIC
    // Error words of all systems (and of the persistent step kernel) copied
    // into host (pinned) memory h[0 .. sys.size()] on the stream, without a
    // synchronisation; status_of reads them once the copies have completed.
    int enqueue_status(int* h);
    int status_of(const int* h) const;
    size_t device_bytes() const;

    void set_stream(cudaStream_t s);
    cudaStream_t stream() const { return stream_; }
    void set_timing(int level);     // 0 off, 1 every kernel, 2 key kernels only
    int kernel_times(int max, const char** names, int64_t* launches, double* ms, int* n);

    std::vector<SysHost*> sys;
    int precision = MD_PREC_SPLIT;
    int64_t launches = 0;

    // instrumentation callbacks (EngineHost)
    void on_rec(const char* name, cudaStream_t s);
    void on_count(int n);

private:
    int capture(GraphRec& g, int kind, bool energy);
    int run_graph(GraphRec& g);
    void drop_graphs();
    void free_tables();
    int ensure_cluster_bufs(SysHost& h, long long need);

    cudaStream_t stream_ = nullptr;
    cudaStream_t own_stream_ = nullptr;
    EngineHost H_;
    SysConst* d_sys_ = nullptr;
    int* d_tile_sys_ = nullptr;
    int* d_item_sys_ = nullptr;
    unsigned* d_hist_ = nullptr;
    unsigned* d_binstart_ = nullptr;
    unsigned* d_cursor_ = nullptr;
    unsigned* d_blocksum_ = nullptr;
    int* d_any_ = nullptr;
    double* d_out_ = nullptr;           // small result buffer
    double* d_clock_ = nullptr;
    unsigned long long* d_seeds_ = nullptr;
    size_t table_bytes_ = 0;

    GraphRec g_step_[2], g_relax_;
    bool timing_ = false;
    int timing_level_ = 0;
    bool capturing_ = false;
    int capture_nodes_ = 0;
    int cond_nodes_ = 0;                    // kernels per run of the conditional rebuild bodies
    GraphRec* cur_rec_ = nullptr;
    cudaStream_t aux_stream_ = nullptr;     // captures the bodies of conditional nodes
    unsigned long long* d_cond_runs_ = nullptr;
    ForceTune* d_tune_ = nullptr;
    PersistCtl* d_pctl_ = nullptr;          // persistent step kernel: barrier, work counter, error flag
    bool persistent_ = false;               // steps run as one persistent launch
    int persistent_mode();                  // recompute persistent_ from the systems' parameters
    double* d_f64part_ = nullptr;
    int* d_f64cnt_ = nullptr;
    int build_step_graph(cudaGraph_t& graph, int kind, bool energy);
    std::map<std::string, std::pair<int64_t, double>> ktimes_;
    std::vector<std::string> korder_;
};

// Eq. (2) screening length (fm) at electron density n_e (fm^-3).
double lambda_thomas_fermi(double n_e);

// Test hook: the nth device allocation from now on fails (0 disarms).
void arm_alloc_failure(long long nth);

// Thread-local error message helpers.
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

}  // namespace pasta
