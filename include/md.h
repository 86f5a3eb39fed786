/*
 * md.h -- C ABI of the B300 (sm_103a) nucleon molecular-dynamics library.
 *
 * Method: Caplan, Schneider, Horowitz & Berry, "Pasta Nucleosynthesis:
 * Molecular dynamics simulations of nuclear statistical equilibrium"
 * (arXiv:1412.8502).  Point protons and neutrons in a periodic cube interact
 * through the Eq. (1) potentials (Table I constants, screening length fixed
 * at 10 fm, Sec. II.A); positions and velocities advance by velocity Verlet,
 * the box side grows as Eq. (3) without rescaling positions, and velocities
 * are rescaled to 3/2 kT per particle every 100 steps (Sec. II.A).  Nuclei
 * are found by the distance-linkage cluster algorithm of Sec. II.C.
 *
 * Conventions for every call:
 *  - Units: fm, MeV, fm/c (c = k_B = 1).
 *  - Return value: MD_OK (0) or a negative MD_E* code; md_last_error()
 *    returns a message for the calling thread's last failure.
 *  - The library owns all device memory.  Host buffers belong to the caller,
 *    who sizes them as documented; the library never keeps a host pointer
 *    after the call returns.
 *  - Particle arrays on the host are particle-major: x[3*i + a] is axis a of
 *    particle i, in the ORIGINAL particle order.  Particles 0 .. Np-1 are
 *    protons and Np .. N-1 neutrons, Np = floor(Yp*N + 0.5).
 *  - There is no CPU fallback: without a usable CUDA device md_create
 *    returns MD_ENODEV.
 *  - A handle may be used by one host thread at a time.
 */
#ifndef PASTA_MD_H
#define PASTA_MD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MD_API __attribute__((visibility("default")))
#else
#define MD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define MD_OK 0
#define MD_EINVAL (-1)    /* invalid argument */
#define MD_ENOMEM (-2)    /* device allocation failed or HBM budget exceeded */
#define MD_ECUDA (-3)     /* a CUDA runtime call failed */
#define MD_ETIMEOUT (-4)  /* a bounded device or host wait gave up */
#define MD_ENUMERIC (-5)  /* a non-finite force or energy was produced */
#define MD_ENODEV (-6)    /* no CUDA device */
#define MD_EAGAIN (-7)    /* md_server_poll: no finished job yet */

#define MD_PREC_SPLIT 0   /* FP32 pair arithmetic, FP64 state and reductions */
#define MD_PREC_FP64 1    /* FP64 everywhere (validation mode) */

typedef struct md_system md_system;
typedef struct md_batch md_batch;
typedef struct md_server md_server;

/* Tunable parameters.  md_params_default() fills the paper's values. */
typedef struct {
    double dt;               /* time step, fm/c (Sec. III: 2 fm/c) */
    double r_nuc;            /* nuclear cutoff, fm (Sec. II.A: 11.5) */
    double r_C;              /* Coulomb cutoff, fm; <= 0 means min(40, L0/2).
                                Must not exceed L0/2 (MD_EINVAL). */
    double lambda_s;         /* Coulomb screening length, fm (Sec. II.A: 10);
                                0 = Thomas-Fermi value of Eq. (2) at the initial
                                proton density (md_lambda_thomas_fermi) */
    double skin;             /* pair-list skin, fm (default 1) */
    int64_t rebuild_every;   /* rebuild pair lists at least every k steps (10) */
    int64_t thermostat_every;/* velocity rescale period in steps (100); 0 = off */
    double T;                /* rescale temperature, MeV (md_create sets it) */
    int32_t precision;       /* MD_PREC_SPLIT (default) or MD_PREC_FP64 */
    int32_t coulomb;         /* screened Coulomb term of V_pp: 0 = off;
                                1 = pairs inside r_C (default, pair lists);
                                2 = every proton pair, nearest image, no cutoff
                                    (Sec. II.A as printed; O(Np^2) per step) */
    double r_pp, r_np;       /* cluster link radii, fm (Sec. II.C: 4.5, 3) */
    int64_t relax_iters;     /* steepest-descent iterations in md_create (500) */
    double relax_gamma;      /* steepest-descent step, fm^2/MeV (0.002) */
    double relax_dmax;       /* per-iteration displacement clamp, fm (0.1) */
    int64_t energy_every;    /* md_step records energies every k steps; 0 = off */
    int32_t sort_bits;       /* spatial-sort bits per axis, 2..7; 0 = from N */
    int32_t affine;          /* 1: scale positions by L_{n+1}/L_n after each box
                                update (an option; the paper does not rescale,
                                Sec. II.A); 0 = off (default) */
    int32_t list_kind;       /* pair lists: 0 = half tile-pair lists (default);
                                1 = per-particle Verlet lists of every pair within
                                its cutoff + skin, rebuilt by the same displacement
                                rule (the paper's neighbour lists, Sec. II.B.1,
                                where skin = delta r = 4 fm).  Split precision
                                only (MD_EINVAL with MD_PREC_FP64). */
    double verlet_pool;      /* list_kind 1: list entries reserved per particle,
                                as a multiple of the expected neighbour count at
                                the initial density (default 2).  A rebuild that
                                needs more makes md_step return MD_ENOMEM. */
    int32_t cond_graph;      /* 1 (default): the rebuild kernels of a step sit in
                                conditional graph nodes and are not launched on
                                steps without a rebuild; 0: plain graph nodes
                                that return at once on such steps (profilers
                                that cannot look inside graphs with conditional
                                nodes).  Results are the same. */
    int32_t force_unroll;    /* split force-pass code: 4 = long unrolled loops
                                (fastest where the far Coulomb field dominates:
                                dense states); 2 = compact, 1 = minimal (fit the
                                instruction cache where several pair classes run
                                at once: clustered, dilute states); 3 = minimal,
                                one warp per block (no warp waits for the others
                                of a block: items of uneven cost); 0 (default) =
                                chosen on the device every 500 steps (from step
                                500 on; the long one before) by timing 4 force
                                passes of each, in engines of at least 131,072
                                nucleons (smaller ones, and persistent steps,
                                run the minimal variant).
                                Results are bitwise the same. */
    int64_t uf_iter_limit;   /* bound on the iterations of every union-find loop
                                of the cluster analyses (a root walk, or the
                                retries of a union), 1 .. 2^31-1 (default 2^26,
                                far above the longest path any input can have).
                                A loop that reaches it gives up and the call
                                returns MD_ETIMEOUT: its labels are then not
                                valid.  No device wait is involved. */
    int64_t wait_limit_ns;   /* bound on each grid-wide wait of the persistent
                                step kernel, ns (default 2e9).  A wait that
                                reaches it gives up, the kernel's blocks leave,
                                and the next md_step / md_batch_step / md_sync
                                returns MD_ETIMEOUT; the state of the systems
                                is then undefined (destroy them). */
    int32_t persistent;      /* each step of all systems of an engine as ONE
                                persistent cooperative launch (phases separated
                                by bounded grid barriers) instead of a graph of
                                separate kernels: 1 = on, 0 = off, -1 (default)
                                = on for batches of two or more systems.  Needs
                                split precision, tile lists and coulomb 0 or 1
                                (MD_EINVAL otherwise when 1; -1 falls back to
                                the graph).  It runs the force-pass code
                                variant force_unroll fixes (0 and 3: the
                                minimal one, its warps in groups of four as
                                every variant there).
                                Results are bitwise those of the graph. */
} md_params;

typedef struct {
    double KE;       /* 1/2 M sum v^2 */
    double PE_nuc;   /* sum over pairs i<j of the nuclear part of Eq. (1) */
    double PE_coul;  /* sum over proton pairs i<j of the screened Coulomb part */
    double virial;   /* sum over pairs i<j of (x_i - x_j) . F_ij */
    double L;        /* box side the energies were evaluated with */
    double t;        /* simulated time, fm/c */
    int64_t step;    /* steps taken since md_create */
    int64_t pairs_nuc;   /* pairs i<j inside r_nuc in that force pass */
    int64_t pairs_coul;  /* proton pairs i<j inside r_C in that pass */
    int64_t candidates;  /* pairs i<j evaluated in that pass, in range or not
                            (md_step_energy only) */
} md_energy_t;

/* State exchange (md_get_state / md_set_state).  The caller owns x, v, f
 * ([N][3] doubles, original order) and type ([N], 1 = proton); any of the
 * four pointers may be NULL on md_get_state to skip that array.
 * L(t) = L_base * (1 + xi_dot * (t - t_base)) is Eq. (3) re-based at t_base.
 * f are the cached forces (MeV/fm) that the next half-kick of velocity
 * Verlet uses, evaluated at x with box side L_F: (x, v, f, L_F) is the whole
 * integrator state, so a state saved with f and loaded with f continues
 * without a fresh force evaluation (in split precision the forces are FP32
 * values, which round-trip exactly through doubles). */
typedef struct {
    int64_t N, Np;
    double* x;
    double* v;
    int8_t* type;
    double L, L_base, t, t_base, xi_dot, L_F;
    int64_t step;
    double* f;
} md_state_view;

typedef struct {
    int64_t n_clusters;      /* clusters (connected proton groups) */
    int64_t n_free;          /* neutrons in no cluster */
    int64_t n_big;           /* clusters with A >= 12 */
    double m_free_n;         /* n_free / N (mass fraction of free neutrons) */
    double A_mean, Z_mean;   /* means over clusters with A >= 12 (0 if none) */
} md_cluster_stats;

typedef struct {
    int64_t N, Np;
    int64_t tiles;           /* 32-particle tiles (proton tiles first) */
    int64_t rebuilds;        /* pair-list rebuilds so far */
    int64_t list_entries;    /* tile pairs in the current force list */
    int64_t launches;        /* kernels launched so far by this handle */
    int64_t device_bytes;    /* device memory owned by this handle */
    int32_t need_wrap;       /* 1 if the box is too small for tile images */
    int32_t sort_bits;
    double tile_halfext_mean;  /* mean / max tile half-extent at the last rebuild, fm */
    double tile_halfext_max;
    int64_t verlet_entries;  /* list_kind 1: neighbour entries (ordered pairs) built
                                at the last rebuild */
    int64_t verlet_slots;    /* list_kind 1: pool slots used (entries + padding of
                                the per-tile blocks) / available */
    int64_t verlet_capacity;
    int32_t force_code;      /* code variant of the split force pass now in use:
                                4 long unrolled loops, 2 compact, 1 minimal,
                                3 minimal in one-warp blocks (md_params
                                force_unroll; 0 there: the device tuner's
                                choice) */
    int32_t pad0;
    int64_t force_trials;    /* trials the device tuner has completed */
} md_info_t;

/* Fill the defaults listed above. */
MD_API void md_params_default(md_params* p);

/* Create a system of N nucleons with proton fraction Yp at density rho
 * (fm^-3) and temperature T (MeV) from `seed`: SplitMix64 uniform positions
 * in the cube of side L0 = cbrt(N/rho), Maxwell velocities rescaled to
 * KE = 3/2 N T with zero total momentum, then params.relax_iters steepest-
 * descent iterations (a reading of the paper's equilibration from random
 * positions, Sec. III.B).  Errors: MD_EINVAL if N < 2, Yp outside [0,1],
 * rho <= 0, T < 0 or r_C > L0/2; MD_ENOMEM; MD_ENODEV; MD_ECUDA. */
MD_API int md_create(int64_t N, double Yp, double rho, double T, uint64_t seed, md_system** out);
/* As md_create with explicit parameters (p may be NULL for defaults). */
MD_API int md_create_ex(int64_t N, double Yp, double rho, double T, uint64_t seed,
                 const md_params* p, md_system** out);
MD_API int md_destroy(md_system* s);

MD_API int md_get_params(const md_system* s, md_params* p);
/* Change parameters between steps (r_C > L0/2 gives MD_EINVAL).  Forces are
 * re-evaluated before the next step. */
MD_API int md_set_params(md_system* s, const md_params* p);
/* Launch on `stream` (a cudaStream_t of the caller's context; NULL = the
 * library's own stream).  The stream must outlive its use by the handle. */
MD_API int md_set_stream(md_system* s, void* stream);

/* Advance n >= 0 velocity-Verlet steps (Sec. II.A) with box growth at
 * expansion rate xi_dot (c/fm, Eq. 3).  When xi_dot differs from the rate
 * in use, Eq. (3) is re-based at the current time so L stays continuous.
 * Synchronises the stream once at the end to report MD_ENUMERIC. */
MD_API int md_step(md_system* s, int64_t n, double xi_dot);
/* As md_step, without the synchronisation: the n steps are enqueued on the
 * handle's stream and the call returns at once.  A non-finite force or a
 * device error is reported by the next md_sync or md_step. */
MD_API int md_step_async(md_system* s, int64_t n, double xi_dot);
/* Wait for the handle's enqueued work; MD_ENUMERIC (or MD_ECUDA) if it
 * failed. */
MD_API int md_sync(md_system* s);

/* Forces of the last force evaluation ([N][3] doubles, original order). */
MD_API int md_forces(md_system* s, double* f_out);

/* Energies of the current state with the current box side (the potential
 * energy is re-evaluated on the device; the cached forces are untouched). */
MD_API int md_energy(md_system* s, md_energy_t* out);
/* Energies recorded by the last md_step that computed them (energy_every);
 * MD_EAGAIN if none was recorded. */
MD_API int md_step_energy(md_system* s, md_energy_t* out);

/* Distance-linkage clusters of Sec. II.C at the current positions.
 * labels [N] (may be NULL): smallest original proton index of the cluster,
 * -1 for a free neutron.  hist_A [N+1], hist_Z [Np+1] (may be NULL): number
 * of clusters with mass number A / charge Z.  Distances are FP64 nearest
 * images; results are exact (bit-identical to a serial FP64 evaluation).
 * The first cluster call of a system allocates its cluster buffers (about
 * 160 B per nucleon, plus the candidate tile lists); MD_ENOMEM if that
 * fails, after which the system stays usable. */
MD_API int md_clusters(md_system* s, int32_t* labels, int64_t* hist_A, int64_t* hist_Z,
                md_cluster_stats* stats);

/* Energy-criterion clusters: the minimum spanning tree in two-particle
 * energy space (MSTE), which Sec. II.C names beside its distance algorithm
 * without defining it.  Reading taken: nucleons i, j are bound when
 *   V_ij(r_ij) + (M/4) |v_i - v_j|^2 < 0,
 * V the pair potential of Eq. (1) at the nearest image (nuclear part inside
 * r_nuc, screened Coulomb for proton pairs as in the force) and (M/4)|dv|^2
 * the kinetic energy of the relative motion; clusters are the connected
 * components of bound pairs.  labels [N] (may be NULL): smallest original
 * index of the cluster (any species); -1 for a neutron bound to nothing; a
 * proton bound to nothing is a cluster by itself.  hist_A [N+1], hist_Z
 * [Np+1] (may be NULL) count clusters by mass and charge (neutron-only
 * clusters in hist_Z[0]); stats as md_clusters.  Decisions are those of
 * FP64 arithmetic in a fixed order (pairs far from the threshold are
 * screened in FP32). */
MD_API int md_clusters_mste(md_system* s, int32_t* labels, int64_t* hist_A, int64_t* hist_Z,
                            md_cluster_stats* stats);

/* Copy the state to the caller (md_state_view above). */
MD_API int md_get_state(md_system* s, md_state_view* view);
/* Replace x, v (and the clock fields) from the caller; N and Np must match,
 * x is wrapped into [0, L).  With f == NULL the forces are re-evaluated at
 * the new state (box side L); otherwise f (evaluated with box side L_F, as
 * md_get_state returns them) become the cached forces and no force pass
 * runs; the state then goes into the system's current particle order, and
 * with the same box side its tiles and pair lists are kept unless the
 * rebuild rule (displacement since the last rebuild, steps since it) asks
 * for new ones: a state saved from the system and loaded back keeps its
 * tiles.  Used for resume and for parity checks. */
MD_API int md_set_state(md_system* s, const md_state_view* view);

MD_API int md_get_info(const md_system* s, md_info_t* info);

/* Per-kernel device timing.  on = 1: md_step records CUDA events around
 * every kernel of each step; on = 2: only around the cell build, the list
 * build, the force pass and the closing kick (fewer event nodes in the step
 * graph); 0: off (MD_EINVAL for other values).  Each call resets the sums.
 * md_kernel_times returns, for up to `max` timed intervals, the name of the
 * kernel that opens it, the count and the summed milliseconds, and the number
 * of intervals available in *n. */
MD_API int md_set_timing(md_system* s, int on);
MD_API int md_kernel_times(md_system* s, int max, const char** names, int64_t* launches,
                    double* ms, int* n);

/* Autotuner: short timed trials (steps each, from the current state, which
 * is restored afterwards) over pair-list skin {0.5, 1, 1.5, 2} fm x spatial-
 * sort resolution, i.e. the cell size of the counting sort, {auto-1, auto,
 * auto+1} bits per axis x (for engines stepping with the persistent kernel
 * and force_unroll 0) the force-pass code variant {long, compact, minimal};
 * keeps the fastest setting and returns the resulting parameters in *chosen
 * (may be NULL).  The tile shape is not a tuning dimension: a tile is one
 * warp's 32 targets (the pair block pairs a 16-source half-warp with two
 * targets per lane).  The physics does not depend on these settings;
 * trajectories differ only by FP32 summation order. */
MD_API int md_autotune(md_system* s, int64_t steps, md_params* chosen);

/* Eq. (2): Thomas-Fermi screening length (fm) of a degenerate relativistic
 * electron gas of density n_e (fm^-3), equal to the proton density. */
MD_API double md_lambda_thomas_fermi(double n_e);

/* Thread-local message describing the last error of this thread. */
MD_API const char* md_last_error(void);

/* Test hook for allocation-failure handling: after md_debug_fail_alloc(n),
 * the n-th device allocation the library makes (1 = the next one), in any
 * thread and through any entry point, fails as if the device were out of
 * memory; the call that made it returns MD_ENOMEM and releases what it had
 * allocated.  n = 0 disarms the hook.  Returns MD_EINVAL for n < 0. */
MD_API int md_debug_fail_alloc(int64_t nth);

/* Cluster analysis (same rules and results as md_clusters) on positions the
 * caller already holds in device memory, for callers that cannot allocate
 * device memory: code running inside another application's memory pool
 * (a foreign allocation breaks its accounting), or loops that must not stall
 * on the allocator.  The paper has no counterpart; this is a service of
 * the library.  It calls no cudaMalloc, cudaFree or allocating routine: its
 * working memory is one fixed file-scope device array, held by every GPU that
 * loads the library until the process exits.
 *   d_x       [N][3] doubles, device, original order, particles 0..Np-1 are
 *             protons; positions inside the periodic cube of side L
 *   d_labels  [N] int32, device (output): smallest proton index of the
 *             cluster, -1 for a free neutron
 *   d_hist_A  [N+1] int64, device (output); d_hist_Z [Np+1] int64 (output)
 *   d_counts  [5] int64, device (output): clusters, free neutrons, clusters
 *             with A >= 12, sum of their A, sum of their Z
 *   stream    cudaStream_t (NULL: legacy default stream); the call is
 *             asynchronous on it.
 * N above 32768 gives MD_EINVAL (fixed scratch limit).  A call whose stream
 * is not capturing looks the scratch array's device address up in the
 * context current at the call (so a device reset or another context on the
 * same device is picked up); a call made under stream capture reuses the
 * address the last uncaptured call on that device found, so make one
 * uncaptured call, in the same context, before capturing (a first call under
 * capture gives MD_EINVAL).  The union-find loops are bounded; if one gives
 * up, d_counts[0] is set to -1 and the labels are not valid.  Calls share the
 * scratch array: two calls whose work overlaps on the GPU race. */
MD_API int md_clusters_noalloc(const double* d_x, int64_t N, int64_t Np, double L, double r_pp, double r_np,
                               int32_t* d_labels, int64_t* d_hist_A, int64_t* d_hist_Z, int64_t* d_counts,
                               void* stream);

/* ---- batched ensemble: many independent systems advanced together ---- */

typedef struct {
    int64_t N;
    double Yp, rho, T;
    uint64_t seed;
    double xi_dot;      /* expansion rate for this job (c/fm) */
    int64_t steps;      /* steps the job asks for (server) */
} md_job;

/* Create n independent systems (md_create semantics per job; p applies to
 * all, NULL for the defaults).  md_batch_step advances all of them: with
 * p->persistent -1 (default) or 1 every step of every system is ONE persistent
 * cooperative kernel launch (its phases separated by grid barriers bounded by
 * p->wait_limit_ns; a barrier that gives up makes the step return
 * MD_ETIMEOUT); with 0, one graph of separate kernels per step.  Each system's
 * trajectory is bitwise the one it has alone.  Errors: MD_EINVAL (n <= 0, a
 * job as md_create rejects, persistent = 1 with FP64, Verlet lists or the
 * all-pairs Coulomb term), MD_ENOMEM, MD_ENODEV, MD_ECUDA. */
MD_API int md_batch_create(int n, const md_job* jobs, const md_params* p, md_batch** out);
MD_API int md_batch_step(md_batch* b, int64_t n);
/* md_autotune for all systems of the batch (one setting shared by all). */
MD_API int md_batch_autotune(md_batch* b, int64_t steps, md_params* chosen);
/* Borrow system i of the batch (owned by the batch; do not destroy). */
MD_API int md_batch_system(md_batch* b, int i, md_system** out);
MD_API int md_batch_destroy(md_batch* b);

/* ---- serving: continuous batching of MD jobs under an HBM budget ---- */

typedef struct {
    int64_t id;
    int32_t status;         /* MD_OK or an error code */
    int32_t reserved0;
    int64_t N, steps;
    md_energy_t energy;     /* energies at the end of the job */
    double wait_ms;         /* submit -> admission */
    double run_ms;          /* admission -> completion */
    double step_p50_ms, step_p99_ms;  /* per-step latency of this job */
} md_result;

MD_API int md_server_create(size_t hbm_budget_bytes, const md_params* p, md_server** out);
/* Queue a job; returns its id.  Thread-safe with respect to poll. */
MD_API int md_server_submit(md_server* sv, const md_job* job, int64_t* id);
/* Pop one finished job (MD_OK) or MD_EAGAIN if none has finished yet. */
MD_API int md_server_poll(md_server* sv, md_result* out);
/* Block until every submitted job has finished (bounded by timeout_s). */
MD_API int md_server_drain(md_server* sv, double timeout_s);
MD_API int md_server_destroy(md_server* sv);

#ifdef __cplusplus
}
#endif
#endif
