// Host engine of the nucleon MD library (see engine.h).
#include "engine.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>

namespace pasta {

// Pool slots for per-particle Verlet lists: verlet_pool x the expected
// number of ordered neighbours within cutoff + skin at the initial density,
// plus one block of 32 x 32 padding slots per tile.
static long long verlet_capacity(int64_t N, int64_t Np, double L0, int T, const md_params& p, double rC) {
    const double V = L0 * L0 * L0, pi = 3.14159265358979323846;
    auto vol = [&](double R) { return std::min(4.0 / 3.0 * pi * R * R * R, V); };
    const double rp = (double)Np / V, rn = (double)(N - Np) / V;
    const double Rn = p.r_nuc + p.skin, Rc = (p.coulomb == 1 ? std::max(rC, p.r_nuc) : p.r_nuc) + p.skin;
    const double per_p = rp * vol(Rc) + rn * vol(Rn), per_n = (rp + rn) * vol(Rn);
    const double expect = (double)Np * per_p + (double)(N - Np) * per_n;
    return (long long)std::ceil(p.verlet_pool * expect) + (long long)T * kTile * kTile;
}

// FP32 pair constants of Eq. (1) for the split-precision force pass.
static PairF pair_consts(const SysConst& c) {
    const double ln2 = 0.69314718055994530942;
    PairF f;
    f.rn2 = (float)(c.r_nuc * c.r_nuc);
    f.rc2 = c.coulomb == 1 ? (float)(c.r_C * c.r_C) : 0.0f;
    f.kq = (float)(-1.0 / (2.0 * c.Lambda * ln2));
    f.A2 = (float)(2.0 * c.a / c.Lambda);
    f.a = (float)c.a;
    f.Ssame = (float)((c.b + c.c) / c.Lambda);
    f.Scross = (float)((c.b - c.c) / c.Lambda);
    f.bsame = (float)(c.b + c.c);
    f.bcross = (float)(c.b - c.c);
    f.kc = (float)(-1.0 / (c.lambda_s * ln2));
    f.l2a = (float)std::log2(c.alpha);
    f.il = (float)(1.0 / c.lambda_s);
    // the force pass tests sources against the box of its targets' current
    // positions, so the radii are the cutoffs plus a rounding margin (no skin)
    const float margin = 2e-3f;
    const float Rn = (float)c.r_nuc + margin, Rc = (float)(c.coulomb == 1 ? c.r_C : 0.0) + margin;
    f.Rn2 = Rn * Rn;
    f.Rc2 = Rc * Rc;
    return f;
}

namespace {
thread_local std::string g_err;

// Allocation-failure injection (md_debug_fail_alloc): when armed with n, the
// n-th device allocation made from then on, in any thread, fails as if the
// device were out of memory.
std::atomic<long long> g_fail_countdown{0};

bool injected_alloc_failure() {
    long long c = g_fail_countdown.load();
    while (c > 0)
        if (g_fail_countdown.compare_exchange_weak(c, c - 1)) return c == 1;
    return false;
}

void rec_cb(void* o, const char* name, cudaStream_t s) { static_cast<Engine*>(o)->on_rec(name, s); }
void count_cb(void* o, int n) { static_cast<Engine*>(o)->on_count(n); }

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(MD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
int dalloc(SysHost& h, T** p, size_t count) {
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    if (injected_alloc_failure())
        return fail(MD_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed (injected)");
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(MD_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    h.allocs.push_back(*p);
    h.bytes += bytes;
    cudaError_t z = cudaMemset(*p, 0, bytes);
    if (z != cudaSuccess) return fail(MD_ECUDA, cudaGetErrorString(z));
    return MD_OK;
}

float __uint_as_float_host(unsigned u) {
    float f;
    std::memcpy(&f, &u, sizeof(f));
    return f;
}

// Sort-grid bits per axis: about 1-2 particles of a species per bin, so the
// bin scan stays small next to the particle traffic while a run of 32
// particles in Hilbert order still spans only ~20 bins.
int auto_bits(int64_t N) {
    int b = (int)std::ceil(std::log2(std::cbrt(0.5 * (double)N)));
    return std::min(7, std::max(2, b));
}
}  // namespace

// Eq. (2): lambda = sqrt(pi)/(2 sqrt(alpha)) (k_F sqrt(k_F^2 + m_e^2))^(-1/2)
// with k_F = (3 pi^2 n_e)^(1/3); hbar = c = 1, lengths in fm, so the electron
// mass enters as m_e c^2 / (hbar c) in fm^-1 and alpha is the fine-structure
// constant.
double lambda_thomas_fermi(double n_e) {
    const double pi = 3.14159265358979323846;
    const double fine = 1.0 / 137.035999084;
    const double m_e = 0.51099895 / 197.3269804;
    const double k_F = std::cbrt(3.0 * pi * pi * n_e);
    return std::sqrt(pi) / (2.0 * std::sqrt(fine)) / std::sqrt(k_F * std::sqrt(k_F * k_F + m_e * m_e));
}

void arm_alloc_failure(long long nth) { g_fail_countdown.store(nth); }

void set_error(const std::string& msg) { g_err = msg; }
int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}
const char* last_error_cstr() { return g_err.c_str(); }

Engine::Engine(int priority) {
    cudaStreamCreateWithPriority(&own_stream_, cudaStreamNonBlocking, priority);
    cudaStreamCreateWithFlags(&aux_stream_, cudaStreamNonBlocking);
    stream_ = own_stream_;
    H_.owner = this;
    H_.rec_fn = rec_cb;
    H_.count_fn = count_cb;
}

Engine::~Engine() {
    cudaStreamSynchronize(stream_);
    drop_graphs();
    for (size_t i = 0; i < sys.size(); ++i) {
        for (void* p : sys[i]->allocs) cudaFree(p);
        delete sys[i];
    }
    sys.clear();
    free_tables();
    if (own_stream_) cudaStreamDestroy(own_stream_);
    if (aux_stream_) cudaStreamDestroy(aux_stream_);
}

void Engine::free_tables() {
    void* ptrs[] = {d_sys_, d_tile_sys_, d_item_sys_, d_hist_, d_binstart_, d_cursor_, d_blocksum_, d_any_, d_out_,
                    d_clock_, d_seeds_, d_cond_runs_, d_tune_, d_f64part_, d_f64cnt_, d_pctl_};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    d_sys_ = nullptr;
    d_tile_sys_ = nullptr;
    d_item_sys_ = nullptr;
    d_hist_ = d_binstart_ = d_cursor_ = d_blocksum_ = nullptr;
    d_any_ = nullptr;
    d_cond_runs_ = nullptr;
    d_tune_ = nullptr;
    d_pctl_ = nullptr;
    d_f64part_ = nullptr;
    d_f64cnt_ = nullptr;
    d_out_ = d_clock_ = nullptr;
    d_seeds_ = nullptr;
    table_bytes_ = 0;
}

void Engine::drop_graphs() {
    GraphRec* gs[] = {&g_step_[0], &g_step_[1], &g_relax_};
    for (GraphRec* g : gs) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        for (cudaEvent_t e : g->events) cudaEventDestroy(e);
        *g = GraphRec();
    }
}

size_t Engine::device_bytes() const {
    size_t b = table_bytes_;
    for (auto* h : sys) b += h->bytes;
    return b;
}

void Engine::set_stream(cudaStream_t s) { stream_ = s ? s : own_stream_; }

void Engine::set_timing(int level) {
    if (level != timing_level_) {
        cudaStreamSynchronize(stream_);
        drop_graphs();
        timing_level_ = level;
        timing_ = level != 0;
    }
    ktimes_.clear();
    korder_.clear();
}

// Level 2 records events only at the start of these kernels (and at the end
// of the step): fewer event nodes in the step graph.
static bool key_kernel(const char* name) {
    static const char* keys[] = {"cell_build", "lists", "force", "force_verlet", "force_fix", "coulomb_pp", "kick"};
    for (const char* k : keys)
        if (std::strcmp(k, name) == 0) return true;
    return false;
}

void Engine::on_rec(const char* name, cudaStream_t s) {
    if (!(capturing_ && timing_ && cur_rec_)) return;
    if (timing_level_ == 2 && !key_kernel(name)) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    cur_rec_->names.push_back(name);
    cur_rec_->events.push_back(e);
}

void Engine::on_count(int n) {
    if (capturing_) capture_nodes_ += n;
    else launches += n;
}

int Engine::kernel_times(int max, const char** names, int64_t* nl, double* ms, int* n) {
    int k = 0;
    for (const std::string& nm : korder_) {
        if (k < max) {
            if (names) names[k] = ktimes_.find(nm)->first.c_str();
            if (nl) nl[k] = ktimes_[nm].first;
            if (ms) ms[k] = ktimes_[nm].second;
        }
        ++k;
    }
    if (n) *n = k;
    return MD_OK;
}

// ------------------------------------------------------------------ systems
int Engine::add_system(int64_t N, double Yp, double rho, double T, uint64_t seed, const md_params& p) {
    if (N < 2 || N > (1ll << 26)) return fail(MD_EINVAL, "N must be in [2, 2^26]");
    if (!(Yp >= 0.0 && Yp <= 1.0)) return fail(MD_EINVAL, "Yp must be in [0, 1]");
    if (!(rho > 0.0)) return fail(MD_EINVAL, "rho must be > 0");
    if (!(T >= 0.0)) return fail(MD_EINVAL, "T must be >= 0");
    if (!(p.dt > 0.0) || !(p.r_nuc > 0.0) || !(p.skin > 0.0) || !(p.lambda_s >= 0.0))
        return fail(MD_EINVAL, "dt, r_nuc, skin must be > 0 and lambda_s >= 0");
    if (p.precision != MD_PREC_SPLIT && p.precision != MD_PREC_FP64) return fail(MD_EINVAL, "bad precision");
    if (p.sort_bits != 0 && (p.sort_bits < 2 || p.sort_bits > 7)) return fail(MD_EINVAL, "sort_bits in 2..7");
    if (p.coulomb < 0 || p.coulomb > 2) return fail(MD_EINVAL, "coulomb must be 0, 1 or 2");
    if (p.affine != 0 && p.affine != 1) return fail(MD_EINVAL, "affine must be 0 or 1");
    if (p.force_unroll < 0 || p.force_unroll > 4)
        return fail(MD_EINVAL, "force_unroll must be 0, 1, 2, 3 or 4");
    if (p.list_kind != 0 && p.list_kind != 1) return fail(MD_EINVAL, "list_kind must be 0 or 1");
    if (p.list_kind == 1 && p.precision != MD_PREC_SPLIT)
        return fail(MD_EINVAL, "Verlet lists (list_kind 1) need split precision");
    if (p.list_kind == 1 && !(p.verlet_pool > 0.0)) return fail(MD_EINVAL, "verlet_pool must be > 0");
    if (p.uf_iter_limit < 1 || p.uf_iter_limit > 0x7fffffff)
        return fail(MD_EINVAL, "uf_iter_limit must be in [1, 2^31 - 1]");
    if (p.persistent < -1 || p.persistent > 1) return fail(MD_EINVAL, "persistent must be -1, 0 or 1");
    if (p.persistent == 1 && (p.precision == MD_PREC_FP64 || p.list_kind != 0 || p.coulomb == 2))
        return fail(MD_EINVAL, "the persistent step needs split precision, tile lists and coulomb 0 or 1");
    if (p.wait_limit_ns < 1) return fail(MD_EINVAL, "wait_limit_ns must be >= 1");
    const double L0 = std::cbrt((double)N / rho);
    double rC = p.r_C > 0.0 ? p.r_C : std::min(40.0, 0.5 * L0);
    // (relative slack of 1e-12 absorbs the rounding of cbrt)
    if (p.coulomb == 1 && rC > 0.5 * L0 * (1.0 + 1e-12)) return fail(MD_EINVAL, "r_C exceeds L0/2");
    if (!sys.empty() && p.precision != precision) return fail(MD_EINVAL, "mixed precision in one engine");
    precision = p.precision;

    auto* h = new SysHost();
    SysHost& s = *h;
    s.N = N;
    s.Np = (int64_t)std::floor(Yp * (double)N + 0.5);
    s.Tp = (int)((s.Np + kTile - 1) / kTile);
    s.T = s.Tp + (int)((N - s.Np + kTile - 1) / kTile);
    s.Tpad = (s.T + kTilesPerBlock - 1) / kTilesPerBlock * kTilesPerBlock;
    s.nbits = p.sort_bits ? p.sort_bits : auto_bits(N);
    s.nbins = 1ll << (3 * s.nbits);
    s.L0 = L0;
    s.rho = rho;
    s.Yp = Yp;
    s.T0 = T;
    s.seed = seed;
    s.prm = p;
    s.prm.r_C = rC;
    s.prm.T = T;
    if (p.lambda_s == 0.0) s.prm.lambda_s = lambda_thomas_fermi((double)s.Np / (L0 * L0 * L0));
    s.xi = 0.0;

    SysConst& c = s.c;
    c.N = (int)N;
    c.Np = (int)s.Np;
    c.T = s.T;
    c.Tp = s.Tp;
    c.nbits = s.nbits;
    c.nbins = s.nbins;
    c.list_cap = (long long)s.T * s.T;
    int rc = MD_OK;
    auto A = [&](auto** ptr, size_t count) {
        if (rc == MD_OK) rc = dalloc(s, ptr, count);
    };
    for (int b = 0; b < 2; ++b) {
        A(&c.x[b], 3 * (size_t)N);
        A(&c.v[b], 3 * (size_t)N);
        A(&c.id[b], (size_t)N);
        A(&c.f32[b], 3 * (size_t)N);
        A(&c.f64[b], 3 * (size_t)N);
    }
    A(&c.disp, 3 * (size_t)N);
    A(&c.key, (size_t)N);
    A(&c.slot, (size_t)N);
    A(&c.xhi, (size_t)s.T * kTile);
    A(&c.xlo, (size_t)s.T * kTile);
    A(&c.torgf, 4 * (size_t)s.T);
    A(&c.thalf, 3 * (size_t)s.T);
    A(&c.sorg, (size_t)(s.T + kTile - 1) / kTile);
    A(&c.shalf, (size_t)(s.T + kTile - 1) / kTile);
    A(&c.lcount, (size_t)s.T);
    A(&c.lnear, (size_t)s.T);
    A(&c.list, (size_t)c.list_cap);
    A(&c.facc, 3 * (size_t)N);
    if (p.list_kind == 1) {
        c.vcap = verlet_capacity(N, s.Np, L0, s.T, p, rC);
        A(&c.vlist, (size_t)c.vcap);
        A(&c.vcount, (size_t)s.T * kTile);
        A(&c.voff, (size_t)s.T);
        A(&c.vwidth, (size_t)s.T);
    }
    A(&c.blk, 4 * (size_t)(s.Tpad / kTilesPerBlock));
    A(&s.d_st, 1);
    A(&s.d_cl, 1);
    A(&s.d_stage, 9 * (size_t)N);
    A(&s.d_stage_t, (size_t)N);
    A(&s.d_stage_lab, (size_t)N);
    if (rc != MD_OK) {
        for (void* q : s.allocs) cudaFree(q);
        delete h;
        return rc;
    }
    c.st = s.d_st;
    c.cl = s.d_cl;
    c.dt = p.dt;
    c.M = 939.0;
    c.hkick = 0.5 * c.dt / c.M;
    c.dtf = (float)c.dt;
    c.T_target = T;
    c.skin = p.skin;
    c.a = 110.0;
    c.b = -26.0;
    c.c = 24.0;
    c.Lambda = 1.25;
    c.lambda_s = s.prm.lambda_s;
    c.affine = p.affine;
    c.alpha = 197.3269804 / 137.035999084;
    c.r_nuc = p.r_nuc;
    c.r_C = rC;
    c.r_pp = p.r_pp;
    c.r_np = p.r_np;
    c.relax_gamma = p.relax_gamma;
    c.relax_dmax = p.relax_dmax;
    c.thermostat_every = (int)p.thermostat_every;
    c.rebuild_every = (int)std::max<int64_t>(1, p.rebuild_every);
    c.coulomb = p.coulomb;
    c.energy_every = (int)p.energy_every;
    c.list_kind = p.list_kind;
    c.force_unroll = p.force_unroll;
    c.uf_limit = (int)p.uf_iter_limit;
    c.pf = pair_consts(c);

    SysState st{};
    st.L = st.L_base = st.L_F = st.L_build = L0;
    st.vscale = 1.0;
    st.xscale = 1.0;
    st.force_rebuild = 1;
    CK(cudaMemcpy(s.d_st, &st, sizeof(st), cudaMemcpyHostToDevice));
    CK(cudaMemset(c.facc, 0, 3 * (size_t)N * sizeof(long long)));   // the force pass expects zeros
    sys.push_back(h);
    return MD_OK;
}

void Engine::remove_system(int idx) {
    cudaStreamSynchronize(stream_);
    SysHost* h = sys[idx];
    for (void* p : h->allocs) cudaFree(p);
    if (h->cl_ready) {
        void* cp[] = {h->hcl.parent, h->hcl.minid, h->hcl.zc, h->hcl.ac, h->hcl.label, h->hcl.hist_A,
                      h->hcl.hist_Z, h->hcl.stats, h->hcl.count, h->hcl.start, h->hcl.list, h->hcl.total};
        for (void* p : cp)
            if (p) cudaFree(p);
    }
    delete h;
    sys.erase(sys.begin() + idx);
}

// Persistent step kernel: wanted by system 0's parameters (1 on, 0 off, -1
// on for two or more systems) and possible for split precision, tile lists
// and the cutoff (or no) Coulomb term in every system.
int Engine::persistent_mode() {
    persistent_ = false;
    if (sys.empty()) return MD_OK;
    const int want = sys[0]->prm.persistent;
    bool ok = precision != MD_PREC_FP64;
    for (SysHost* h : sys) ok = ok && h->c.list_kind == 0 && h->c.coulomb != 2;
    if (want == 1 && !ok)
        return fail(MD_EINVAL, "the persistent step needs split precision, tile lists and coulomb 0 or 1");
    persistent_ = ok && (want == 1 || (want == -1 && sys.size() > 1));
    if (persistent_ && prepare_step_persistent() != 0) {
        const cudaError_t e = cudaGetLastError();
        return fail(MD_ECUDA, std::string("persistent step kernel: ") + cudaGetErrorString(e));
    }
    return MD_OK;
}

// Force-pass variant of the launches that do not select it per step: the one
// force_unroll fixes, else the long one in engines where the device tuner runs
// (large ones: it times the others) and the minimal one where it does not
// (small engines and persistent steps, which mostly run dilute or mixed
// systems; over the 51,200 expansion the minimal variant measured 260 M
// against 240 M nucleon-steps/s with the long one, 1.5% slower only in the
// dense first 1,000 steps).
static int fixed_variant(int fu, bool tuner) {
    return fu == 4 ? 0 : fu == 2 ? 1 : fu == 1 ? 2 : fu == 3 ? 3 : (tuner ? 0 : 2);
}

int Engine::build_tables() {
    cudaStreamSynchronize(stream_);
    drop_graphs();
    free_tables();
    const int n = (int)sys.size();
    int tiles = 0, items = 0;
    long long bins = 0;
    for (SysHost* h : sys) {
        h->c.tile_base = tiles;
        h->c.bin_base = bins;
        h->c.item_base = items;
        h->c.n_items = sys_items(h->c.T, h->c.Tp);
        tiles += h->Tpad;
        items += (h->c.n_items + 3) / 4 * 4;
        bins += 2 * h->nbins;
    }
    if (tiles == 0) tiles = kTilesPerBlock;
    if (items == 0) items = 4;
    if (bins == 0) bins = 1;
    std::vector<int> ts(tiles, -1), is(items, -1);
    for (int s = 0; s < n; ++s) {
        for (int t = 0; t < sys[s]->Tpad; ++t) ts[sys[s]->c.tile_base + t] = s;
        for (int v = 0; v < (sys[s]->c.n_items + 3) / 4 * 4; ++v) is[sys[s]->c.item_base + v] = s;
    }
    const int nscan = (int)((bins + 8191) / 8192);
    auto A = [&](auto** p, size_t bytes) -> int {
        if (injected_alloc_failure()) return fail(MD_ENOMEM, "engine table allocation failed (injected)");
        cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(bytes, 16));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(MD_ENOMEM, "engine table allocation failed");
        }
        cudaMemset(*p, 0, std::max<size_t>(bytes, 16));
        table_bytes_ += bytes;
        return MD_OK;
    };
    int rc = MD_OK;
    if ((rc = A(&d_sys_, sizeof(SysConst) * std::max(n, 1)))) return rc;
    if ((rc = A(&d_tile_sys_, sizeof(int) * tiles))) return rc;
    if ((rc = A(&d_item_sys_, sizeof(int) * items))) return rc;
    if ((rc = A(&d_hist_, sizeof(unsigned) * bins))) return rc;
    if ((rc = A(&d_binstart_, sizeof(unsigned) * bins))) return rc;
    if ((rc = A(&d_cursor_, sizeof(unsigned) * bins))) return rc;
    if ((rc = A(&d_blocksum_, sizeof(unsigned) * (nscan + 1)))) return rc;
    if ((rc = A(&d_any_, sizeof(int)))) return rc;
    if ((rc = A(&d_cond_runs_, sizeof(unsigned long long)))) return rc;
    if ((rc = A(&d_tune_, sizeof(ForceTune)))) return rc;
    if ((rc = A(&d_pctl_, sizeof(PersistCtl)))) return rc;
    // FP64 mode: split the tiles' entries over blocks while tiles < SMs
    int sms = 148, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int chunks = precision == MD_PREC_FP64 ? std::max(1, std::min(8, sms / std::max(tiles, 1))) : 1;
    if (chunks > 1) {
        if ((rc = A(&d_f64part_, sizeof(double) * 3 * (size_t)chunks * tiles * kTile))) return rc;
        if ((rc = A(&d_f64cnt_, sizeof(int) * tiles))) return rc;
    }
    if ((rc = A(&d_out_, sizeof(double) * 16))) return rc;
    if ((rc = A(&d_clock_, sizeof(double) * 8))) return rc;
    if ((rc = A(&d_seeds_, sizeof(unsigned long long) * std::max(n, 1)))) return rc;
    std::vector<SysConst> hs(n);
    for (int s = 0; s < n; ++s) hs[s] = sys[s]->c;
    if (n) CK(cudaMemcpy(d_sys_, hs.data(), sizeof(SysConst) * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_tile_sys_, ts.data(), sizeof(int) * tiles, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_item_sys_, is.data(), sizeof(int) * items, cudaMemcpyHostToDevice));
    EngineDev& E = H_.dev;
    E.sys = d_sys_;
    E.tile_sys = d_tile_sys_;
    E.item_sys = d_item_sys_;
    E.nitems = items;
    E.nsys = n;
    E.ntiles = tiles;
    E.nbins_total = bins;
    E.hist = d_hist_;
    E.binstart = d_binstart_;
    E.cursor = d_cursor_;
    E.blocksum = d_blocksum_;
    E.any_rebuild = d_any_;
    E.cond_runs = d_cond_runs_;
    E.tune = d_tune_;
    E.f64chunks = chunks;
    E.f64part = d_f64part_;
    E.f64cnt = d_f64cnt_;
    long long ntot = 0;
    for (SysHost* h : sys) ntot += h->N;
    if ((rc = persistent_mode())) return rc;
    E.tune_variants = (precision != MD_PREC_FP64 && ntot >= kVariantMinN && !persistent_) ? 1 : 0;
    {
        const int fu = sys.empty() ? 0 : (int)sys[0]->prm.force_unroll;
        H_.fixed_var = fixed_variant(fu, E.tune_variants != 0);
    }
    H_.precision = precision;
    H_.any_pp = false;
    H_.any_verlet = false;
    for (SysHost* h : sys) {
        H_.any_pp |= (h->c.coulomb == 2);
        H_.any_verlet |= (h->c.list_kind == 1);
    }
    return MD_OK;
}

int Engine::initialise() {
    int rc = initialise_async();
    if (rc) return rc;
    return check_errors();
}

int Engine::initialise_async(bool relax) {
    std::vector<unsigned long long> seeds;
    for (SysHost* h : sys) seeds.push_back(h->seed);
    CK(cudaMemcpyAsync(d_seeds_, seeds.data(), sizeof(unsigned long long) * seeds.size(), cudaMemcpyHostToDevice,
                       stream_));
    launch_init(H_, stream_, d_seeds_);
    CK(cudaGetLastError());
    int rc = refresh(-1);
    if (rc) return rc;
    return relax ? relax_async(relax_iters()) : MD_OK;
}

int64_t Engine::relax_iters() const {
    int64_t iters = 0;
    for (const SysHost* h : sys) iters = std::max(iters, h->prm.relax_iters);
    return iters;
}

int Engine::relax_async(int64_t n) {
    int rc;
    if (n > 0 && !g_relax_.exec && (rc = capture(g_relax_, 1, false))) return rc;
    for (int64_t k = 0; k < n; ++k)
        if ((rc = run_graph(g_relax_))) return rc;
    return MD_OK;
}

// ------------------------------------------------------------------ graphs
// A step (kind 0) or relaxation iteration (kind 1) as one graph: kick-drift
// (or the steepest-descent update) and the rebuild decision, the rebuild
// kernels in two conditional (IF) nodes on handles that the decision kernel
// sets (on steps without a rebuild they are not launched), then the forces
// and the closing kick.  The plain segments are captured into the graph from
// its current frontier; the conditional nodes are added between them and
// their bodies captured on a second stream.  Timing events (not allowed
// inside conditional bodies) bracket each conditional node.
int Engine::capture(GraphRec& g, int kind, bool energy) {
    g = GraphRec();
    capturing_ = true;
    capture_nodes_ = 0;
    // kernels of the conditional rebuild bodies (the same in every graph
    // that has them; a persistent step graph has none and keeps the count)
    const int prev_cond = cond_nodes_;
    cond_nodes_ = 0;
    cur_rec_ = &g;
    cudaGraph_t graph = nullptr;
    int rc = build_step_graph(graph, kind, energy);
    if (cond_nodes_ == 0) cond_nodes_ = prev_cond;
    capturing_ = false;
    cur_rec_ = nullptr;
    if (rc != MD_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(MD_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    g.nodes = capture_nodes_;
    g.cond_nodes = cond_nodes_;
    return MD_OK;
}

int Engine::build_step_graph(cudaGraph_t& graph, int kind, bool energy) {
    CK(cudaGraphCreate(&graph, 0));
    // one handle per conditional node (a graph may not hold a handle without
    // its node): the two rebuild IF nodes and, in split precision, the SWITCH
    // node of the force-pass code variant
    const bool cond = sys.empty() || sys[0]->prm.cond_graph != 0;
    const bool split = precision != MD_PREC_FP64;
    const bool multi = split && H_.dev.tune_variants;     // the step selects the force-pass variant
    // otherwise the variant md_params.force_unroll fixes (0: see fixed_variant)
    const int fu = sys.empty() ? 0 : (int)sys[0]->prm.force_unroll;
    const int fixed_var = fixed_variant(fu, H_.dev.tune_variants != 0);
    if (kind == 0 && persistent_) {
        // the whole step of every system: one persistent launch
        CK(cudaStreamBeginCaptureToGraph(stream_, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        const int lr = launch_step_persistent(H_, stream_, energy, fixed_var, d_pctl_,
                                              (unsigned long long)sys[0]->prm.wait_limit_ns);
        if (timing_) {
            cudaEvent_t ev;
            cudaEventCreate(&ev);
            cudaEventRecordWithFlags(ev, stream_, cudaEventRecordExternal);
            cur_rec_->events.push_back(ev);
        }
        const cudaError_t le = cudaGetLastError();
        cudaGraph_t out = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(stream_, &out);
        if (lr != 0 || le != cudaSuccess || e2 != cudaSuccess)
            return fail(MD_ECUDA, std::string("persistent step launch: ") +
                                      cudaGetErrorString(le != cudaSuccess ? le : e2));
        return MD_OK;
    }
    cudaGraphConditionalHandle h[3] = {0, 0, 0};
    if (cond) {
        for (int k = 0; k < 2; ++k) CK(cudaGraphConditionalHandleCreate(&h[k], graph, 0, cudaGraphCondAssignDefault));
        if (multi) CK(cudaGraphConditionalHandleCreate(&h[2], graph, 0, cudaGraphCondAssignDefault));
    }
    std::vector<cudaGraphNode_t> front;
    int rc;
    // segment: launches captured into `graph` after the frontier, which then moves
    auto segment = [&](auto&& launches) -> int {
        CK(cudaStreamBeginCaptureToGraph(stream_, graph, front.empty() ? nullptr : front.data(), nullptr,
                                         front.size(), cudaStreamCaptureModeThreadLocal));
        launches();
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        cudaError_t e = cudaStreamGetCaptureInfo(stream_, &cs, nullptr, nullptr, &deps, nullptr, &nd);
        std::vector<cudaGraphNode_t> next(deps, deps + (e == cudaSuccess ? nd : 0));
        cudaGraph_t out = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(stream_, &out);
        if (e != cudaSuccess || e2 != cudaSuccess)
            return fail(MD_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
        front.swap(next);
        return MD_OK;
    };
    // conditional node after the frontier; its body captured on the second stream
    auto conditional = [&](int part) -> int {
        cudaGraphNodeParams p = {};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = h[part];
        p.conditional.type = cudaGraphCondTypeIf;
        p.conditional.size = 1;
        cudaGraphNode_t node;
        CK(cudaGraphAddNode(&node, graph, front.empty() ? nullptr : front.data(), nullptr, front.size(), &p));
        CK(cudaStreamBeginCaptureToGraph(aux_stream_, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal));
        const int n0 = capture_nodes_;
        if (part == 0) launch_cell_build(H_, aux_stream_, false);
        else launch_list_build(H_, aux_stream_, false);
        cond_nodes_ += capture_nodes_ - n0;
        capture_nodes_ = n0;
        cudaGraph_t body = nullptr;
        CK(cudaStreamEndCapture(aux_stream_, &body));
        front.assign(1, node);
        return MD_OK;
    };
    // SWITCH node after the frontier: body v launches force-pass variant v
    auto variant_switch = [&]() -> int {
        cudaGraphNodeParams p = {};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = h[2];
        p.conditional.type = cudaGraphCondTypeSwitch;
        p.conditional.size = kVariants;
        cudaGraphNode_t node;
        CK(cudaGraphAddNode(&node, graph, front.empty() ? nullptr : front.data(), nullptr, front.size(), &p));
        const int n0 = capture_nodes_;
        for (int v = 0; v < kVariants; ++v) {
            CK(cudaStreamBeginCaptureToGraph(aux_stream_, p.conditional.phGraph_out[v], nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal));
            launch_force_variant(H_, aux_stream_, kind == 0 && energy, -1, v, false);
            cudaGraph_t body = nullptr;
            CK(cudaStreamEndCapture(aux_stream_, &body));
        }
        capture_nodes_ = n0 + 1;           // one variant runs every step
        front.assign(1, node);
        return MD_OK;
    };
    // split precision steps convert the force accumulators in the closing kick
    // (not with the all-pairs Coulomb term, which adds to the converted forces)
    const bool fuse = split && kind == 0 && !H_.any_pp;
    // the closing part of a step: kick, finalisation
    auto closing = [&]() {
        if (kind == 0) launch_kick_finalize(H_, stream_, energy, fuse);
        if (timing_) {
            cudaEvent_t ev;
            cudaEventCreate(&ev);
            cudaEventRecordWithFlags(ev, stream_, cudaEventRecordExternal);
            cur_rec_->events.push_back(ev);
        }
    };
    const bool fe = kind == 0 && energy;
    if (!cond) {
        // plain nodes: the rebuild kernels return at once unless a system rebuilds
        rc = segment([&] {
            if (kind == 0) launch_kick_drift(H_, stream_);
            else launch_sd_update(H_, stream_);
            launch_decide(H_, stream_, 0, -1, 0, 0, false, 0, false);
            H_.rec("cell_build", stream_);
            launch_cell_build(H_, stream_, false);
            H_.rec("lists", stream_);
            launch_list_build(H_, stream_, false);
        });
        if (rc) return rc;
        // all force-pass variants (all but one return at once), or the fixed one
        return segment([&] {
            if (split) {
                launch_force_pre(H_, stream_, fe, -1, false);
                if (multi)
                    for (int v = 0; v < kVariants; ++v) launch_force_variant(H_, stream_, fe, -1, v, true);
                else
                    launch_force_variant(H_, stream_, fe, -1, fixed_var, false);
                launch_force_post(H_, stream_, fe, -1, 0, !fuse);
            } else {
                launch_force(H_, stream_, fe, -1, 0);
            }
            closing();
        });
    } else {
        if ((rc = segment([&] {
                 if (kind == 0) launch_kick_drift(H_, stream_);
                 else launch_sd_update(H_, stream_);
                 launch_decide(H_, stream_, 0, -1, h[0], h[1], true, h[2], multi);
                 H_.rec("cell_build", stream_);
             })))
            return rc;
        if ((rc = conditional(0))) return rc;
        if ((rc = segment([&] { H_.rec("lists", stream_); }))) return rc;
        if ((rc = conditional(1))) return rc;
    }
    if (!split) return segment([&] {
        launch_force(H_, stream_, fe, -1, 0);
        closing();
    });
    if (!multi) return segment([&] {
        launch_force_pre(H_, stream_, fe, -1, false);
        launch_force_variant(H_, stream_, fe, -1, fixed_var, false);
        launch_force_post(H_, stream_, fe, -1, 0, !fuse);
        closing();
    });
    if ((rc = segment([&] { launch_force_pre(H_, stream_, fe, -1, false); }))) return rc;
    if ((rc = variant_switch())) return rc;
    return segment([&] {
        launch_force_post(H_, stream_, fe, -1, 0, !fuse);
        closing();
    });
}

int Engine::run_graph(GraphRec& g) {
    CK(cudaGraphLaunch(g.exec, stream_));
    launches += g.nodes;
    if (timing_ && g.events.size() > 1) {
        CK(cudaStreamSynchronize(stream_));
        for (size_t i = 0; i + 1 < g.events.size(); ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, g.events[i], g.events[i + 1]);
            auto it = ktimes_.find(g.names[i]);
            if (it == ktimes_.end()) {
                korder_.push_back(g.names[i]);
                it = ktimes_.emplace(g.names[i], std::make_pair((int64_t)0, 0.0)).first;
            }
            it->second.first += 1;
            it->second.second += ms;
        }
    }
    return MD_OK;
}

// ------------------------------------------------------------------ ops
int Engine::refresh(int only) {
    launch_rebuild(H_, stream_, 1, only);
    launch_force(H_, stream_, false, only, 0);
    launch_mark_forces(H_, stream_, only);       // the forces' box side is the current one
    CK(cudaGetLastError());
    for (size_t s = 0; s < sys.size(); ++s)
        if (only < 0 || (int)s == only) sys[s]->dirty = false;
    return MD_OK;
}

int Engine::check_errors() {
    const int n = (int)sys.size();
    std::vector<int> errs(n, 0);
    for (int s = 0; s < n; ++s)
        CK(cudaMemcpyAsync(&errs[s], &sys[s]->d_st->error, sizeof(int), cudaMemcpyDeviceToHost, stream_));
    int perr = 0;
    if (d_pctl_) CK(cudaMemcpyAsync(&perr, &d_pctl_->error, sizeof(int), cudaMemcpyDeviceToHost, stream_));
    CK(cudaStreamSynchronize(stream_));
    if (perr) {
        CK(cudaMemsetAsync(&d_pctl_->error, 0, sizeof(int), stream_));
        CK(cudaStreamSynchronize(stream_));
        return fail(MD_ETIMEOUT, "a grid-wide wait of the persistent step kernel gave up (wait_limit_ns); "
                                 "the state of the systems is undefined");
    }
    for (int s = 0; s < n; ++s) {
        if (errs[s] & 4)
            return fail(MD_ENOMEM, "Verlet list pool of system " + std::to_string(s) +
                                       " exhausted at a rebuild (raise verlet_pool)");
        if (errs[s]) return fail(MD_ENUMERIC, "non-finite force in system " + std::to_string(s));
    }
    return MD_OK;
}

int Engine::enqueue_status(int* h) {
    const int n = (int)sys.size();
    for (int s = 0; s < n; ++s)
        CK(cudaMemcpyAsync(&h[s], &sys[s]->d_st->error, sizeof(int), cudaMemcpyDeviceToHost, stream_));
    h[n] = 0;
    if (d_pctl_) CK(cudaMemcpyAsync(&h[n], &d_pctl_->error, sizeof(int), cudaMemcpyDeviceToHost, stream_));
    return MD_OK;
}

int Engine::status_of(const int* h) const {
    const int n = (int)sys.size();
    if (h[n]) return fail(MD_ETIMEOUT, "a grid-wide wait of the persistent step kernel gave up (wait_limit_ns)");
    for (int s = 0; s < n; ++s) {
        if (h[s] & 4) return fail(MD_ENOMEM, "Verlet list pool of system " + std::to_string(s) + " exhausted");
        if (h[s]) return fail(MD_ENUMERIC, "non-finite force in system " + std::to_string(s));
    }
    return MD_OK;
}

int Engine::step(int64_t n, const std::vector<double>* xi) {
    int rc = step_async(n, xi, nullptr);
    if (rc) return rc;
    return check_errors();
}

size_t Engine::estimate_bytes(int64_t N, double Yp, double rho, const md_params& p) {
    const int64_t Np = (int64_t)std::floor(Yp * (double)N + 0.5);
    const int64_t T = (Np + kTile - 1) / kTile + (N - Np + kTile - 1) / kTile;
    const int64_t Tpad = (T + kTilesPerBlock - 1) / kTilesPerBlock * kTilesPerBlock;
    const int nbits = p.sort_bits ? p.sort_bits : auto_bits(N);
    const int64_t nb = 2ll << (3 * nbits);
    size_t b = 0;
    b += 2 * (size_t)N * (8 * 3 + 8 * 3 + 4 + 4 * 3 + 8 * 3);   // x, v, id, f32, f64
    b += (size_t)N * (4 * 3 + 4 + 4 + 9 * 8 + 1 + 4 + 8 * 3);   // disp, key, slot, staging, facc
    b += (size_t)T * (32 * 32 + 8 * 3 + 16 + 12 + 4 + 4) + 64 * (size_t)sys_items((int)T, (int)((Np + kTile - 1) / kTile)) +
         4 * 8 * Tpad;
    b += (size_t)T * T * 4;                                      // pair list
    b += (size_t)nb * 12 + 4096;                                 // engine bins
    if (p.list_kind == 1) {
        const double L0 = std::cbrt((double)N / rho);
        const double rC = p.r_C > 0.0 ? p.r_C : std::min(40.0, 0.5 * L0);
        b += 4 * (size_t)verlet_capacity(N, Np, L0, (int)T, p, rC) + (size_t)T * (32 * 4 + 12);
    }
    return b;
}

int Engine::step_async(int64_t n, const std::vector<double>* xi, cudaEvent_t* events) {
    if (n < 0) return fail(MD_EINVAL, "n must be >= 0");
    int rc;
    bool any_dirty = false;
    for (SysHost* h : sys) any_dirty |= h->dirty;
    if (any_dirty) {
        for (size_t s = 0; s < sys.size(); ++s) {
            if (!sys[s]->dirty) continue;
            int one = 1;
            CK(cudaMemcpyAsync(&sys[s]->d_st->force_rebuild, &one, sizeof(int), cudaMemcpyHostToDevice, stream_));
            if ((rc = refresh((int)s))) return rc;
        }
    }
    if (xi) {
        for (size_t s = 0; s < sys.size(); ++s) {
            const double x = (*xi)[s];
            if (x != sys[s]->xi) {
                launch_set_rate(H_, stream_, (int)s, x);
                sys[s]->xi = x;
            }
        }
    }
    const int64_t ee = sys.empty() ? 0 : sys[0]->prm.energy_every;
    for (int64_t k = 0; k < n; ++k) {
        const int64_t next = sys.empty() ? 0 : sys[0]->host_step + 1;
        const int e = (ee > 0 && next % ee == 0) ? 1 : 0;
        if (!g_step_[e].exec && (rc = capture(g_step_[e], 0, e == 1))) return rc;
        if (events) CK(cudaEventRecord(events[k], stream_));
        if ((rc = run_graph(g_step_[e]))) return rc;
        for (SysHost* h : sys) h->host_step += 1;
    }
    if (events) CK(cudaEventRecord(events[n], stream_));
    CK(cudaGetLastError());
    return MD_OK;
}

int Engine::forces(int idx, double* f_out) {
    SysHost& h = *sys[idx];
    int rc;
    if (h.dirty && (rc = refresh(idx))) return rc;
    double* d_f = h.d_stage + 6 * h.N;
    launch_gather(H_, stream_, idx, nullptr, nullptr, d_f, nullptr);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(f_out, d_f, sizeof(double) * 3 * h.N, cudaMemcpyDeviceToHost, stream_));
    CK(cudaStreamSynchronize(stream_));
    return MD_OK;
}

int Engine::energy(int idx, md_energy_t* e) {
    SysHost& h = *sys[idx];
    int rc;
    if (h.dirty && (rc = refresh(idx))) return rc;
    launch_energy_now(H_, stream_, idx, d_out_);
    CK(cudaGetLastError());
    double o[9];
    CK(cudaMemcpyAsync(o, d_out_, sizeof(o), cudaMemcpyDeviceToHost, stream_));
    CK(cudaStreamSynchronize(stream_));
    e->KE = o[0];
    e->PE_nuc = o[1];
    e->PE_coul = o[2];
    e->virial = o[3];
    e->L = o[4];
    e->t = o[5];
    e->step = (int64_t)o[6];
    e->pairs_nuc = (int64_t)o[7];
    e->pairs_coul = (int64_t)o[8];
    return check_errors();
}

int Engine::step_energy(int idx, md_energy_t* e) {
    SysState st;
    CK(cudaMemcpyAsync(&st, sys[idx]->d_st, sizeof(st), cudaMemcpyDeviceToHost, stream_));
    CK(cudaStreamSynchronize(stream_));
    if (!st.have_energy) return fail(MD_EAGAIN, "no energies recorded (energy_every = 0?)");
    e->KE = st.KE;
    e->PE_nuc = st.PE_nuc;
    e->PE_coul = st.PE_coul;
    e->virial = st.virial;
    e->L = st.e_L;
    e->t = st.e_t;
    e->step = st.e_step;
    e->pairs_nuc = st.e_pairs_nuc;
    e->pairs_coul = st.e_pairs_coul;
    e->candidates = st.e_cand;
    return MD_OK;
}

int Engine::ensure_cluster_bufs(SysHost& h, long long need) {
    ClusterBufs& B = h.hcl;
    int rc = MD_OK;
    if (!h.cl_ready) {
        std::memset(&B, 0, sizeof(B));
        auto A = [&](auto** p, size_t count) {
            if (rc == MD_OK) rc = dalloc(h, p, count);
        };
        A(&B.parent, (size_t)h.N);
        A(&B.minid, (size_t)h.N);
        A(&B.zc, (size_t)h.N);
        A(&B.ac, (size_t)h.N);
        A(&B.label, (size_t)h.N);
        A(&B.hist_A, (size_t)h.N + 1);
        A(&B.hist_Z, (size_t)h.Np + 1);
        A(&B.stats, 8);
        A(&B.count, (size_t)h.T);
        A(&B.start, (size_t)h.T + 1);
        A(&B.total, 1);
        // links: about 6 per proton for the distance clusters in the dense
        // start, 12 inside nuclei at saturation density (the energy-criterion
        // clusters link all species); beyond the capacity the link pass unites
        // the pair itself
        B.ecap = std::max<long long>(16 * (long long)h.N, 1024);
        A(&B.edges, (size_t)B.ecap);
        if (rc) return rc;
        h.cl_ready = true;
    }
    if (need > B.cap) {
        long long cap = std::max<long long>(need + need / 4, 1024);
        int* nl = nullptr;
        if ((rc = dalloc(h, &nl, (size_t)cap))) return rc;
        B.list = nl;   // the previous list stays allocated until the system is freed
        B.cap = cap;
    }
    CK(cudaMemcpyAsync(h.d_cl, &B, sizeof(B), cudaMemcpyHostToDevice, stream_));
    return MD_OK;
}

int Engine::clusters(int idx, int32_t* labels, int64_t* hA, int64_t* hZ, md_cluster_stats* out) {
    SysHost& h = *sys[idx];
    int rc;
    if (h.dirty && (rc = refresh(idx))) return rc;
    if ((rc = ensure_cluster_bufs(h, 0))) return rc;
    launch_cluster_lists(H_, stream_, 0, idx);
    long long total = 0;
    CK(cudaMemcpyAsync(&total, h.hcl.total, sizeof(total), cudaMemcpyDeviceToHost, stream_));
    CK(cudaStreamSynchronize(stream_));
    if ((rc = ensure_cluster_bufs(h, total))) return rc;
    launch_cluster_lists(H_, stream_, 1, idx);
    launch_clusters(H_, stream_, idx, (int)h.Np, (int)h.N, h.Tp, h.T, h.d_stage_lab);
    CK(cudaGetLastError());
    long long st[8];
    if (labels)
        CK(cudaMemcpyAsync(labels, h.d_stage_lab, sizeof(int32_t) * h.N, cudaMemcpyDeviceToHost, stream_));
    if (hA) CK(cudaMemcpyAsync(hA, h.hcl.hist_A, sizeof(int64_t) * (h.N + 1), cudaMemcpyDeviceToHost, stream_));
    if (hZ) CK(cudaMemcpyAsync(hZ, h.hcl.hist_Z, sizeof(int64_t) * (h.Np + 1), cudaMemcpyDeviceToHost, stream_));
    CK(cudaMemcpyAsync(st, h.hcl.stats, sizeof(st), cudaMemcpyDeviceToHost, stream_));
    CK(cudaStreamSynchronize(stream_));
    if (st[7])
        return fail(MD_ETIMEOUT, "a union-find loop reached uf_iter_limit (" + std::to_string(h.prm.uf_iter_limit) +
                                     " iterations); the cluster labels are not valid");
    if (out) {
        out->n_clusters = st[0];
        out->n_free = st[1];
        out->n_big = st[2];
        out->m_free_n = (double)st[1] / (double)h.N;
        out->A_mean = st[2] ? (double)st[3] / (double)st[2] : 0.0;
        out->Z_mean = st[2] ? (double)st[4] / (double)st[2] : 0.0;
    }
    return MD_OK;
}

int Engine::clusters_mste(int idx, int32_t* labels, int64_t* hA, int64_t* hZ, md_cluster_stats* out) {
    SysHost& h = *sys[idx];
    int rc;
    if (h.dirty && (rc = refresh(idx))) return rc;
    if ((rc = ensure_cluster_bufs(h, 0))) return rc;
    launch_mste(H_, stream_, idx, (int)h.N, h.T, h.d_stage_lab);
    CK(cudaGetLastError());
    long long st[8];
    if (labels)
        CK(cudaMemcpyAsync(labels, h.d_stage_lab, sizeof(int32_t) * h.N, cudaMemcpyDeviceToHost, stream_));
    if (hA) CK(cudaMemcpyAsync(hA, h.hcl.hist_A, sizeof(int64_t) * (h.N + 1), cudaMemcpyDeviceToHost, stream_));
    if (hZ) CK(cudaMemcpyAsync(hZ, h.hcl.hist_Z, sizeof(int64_t) * (h.Np + 1), cudaMemcpyDeviceToHost, stream_));
    CK(cudaMemcpyAsync(st, h.hcl.stats, sizeof(st), cudaMemcpyDeviceToHost, stream_));
    CK(cudaStreamSynchronize(stream_));
    if (st[7])
        return fail(MD_ETIMEOUT, "a union-find loop reached uf_iter_limit (" + std::to_string(h.prm.uf_iter_limit) +
                                     " iterations); the cluster labels are not valid");
    if (out) {
        out->n_clusters = st[0];
        out->n_free = st[1];
        out->n_big = st[2];
        out->m_free_n = (double)st[1] / (double)h.N;
        out->A_mean = st[2] ? (double)st[3] / (double)st[2] : 0.0;
        out->Z_mean = st[2] ? (double)st[4] / (double)st[2] : 0.0;
    }
    return MD_OK;
}

int Engine::get_state(int idx, md_state_view* v) {
    SysHost& h = *sys[idx];
    int rc;
    if (v->f && h.dirty && (rc = refresh(idx))) return rc;
    double* dx = h.d_stage;
    double* dv = h.d_stage + 3 * h.N;
    double* df = h.d_stage + 6 * h.N;
    launch_gather(H_, stream_, idx, v->x ? dx : nullptr, v->v ? dv : nullptr, v->f ? df : nullptr,
                  v->type ? h.d_stage_t : nullptr);
    CK(cudaGetLastError());
    if (v->x) CK(cudaMemcpyAsync(v->x, dx, sizeof(double) * 3 * h.N, cudaMemcpyDeviceToHost, stream_));
    if (v->v) CK(cudaMemcpyAsync(v->v, dv, sizeof(double) * 3 * h.N, cudaMemcpyDeviceToHost, stream_));
    if (v->f) CK(cudaMemcpyAsync(v->f, df, sizeof(double) * 3 * h.N, cudaMemcpyDeviceToHost, stream_));
    if (v->type) CK(cudaMemcpyAsync(v->type, h.d_stage_t, h.N, cudaMemcpyDeviceToHost, stream_));
    SysState st;
    CK(cudaMemcpyAsync(&st, h.d_st, sizeof(st), cudaMemcpyDeviceToHost, stream_));
    CK(cudaStreamSynchronize(stream_));
    v->N = h.N;
    v->Np = h.Np;
    v->L = st.L;
    v->L_base = st.L_base;
    v->t = st.t;
    v->t_base = st.t_base;
    v->xi_dot = st.xi_dot;
    v->L_F = st.L_F;
    v->step = st.step;
    return MD_OK;
}

int Engine::set_state(int idx, const md_state_view* v) {
    SysHost& h = *sys[idx];
    if (v->N != h.N || v->Np != h.Np) return fail(MD_EINVAL, "N / Np do not match the system");
    if (!v->x || !v->v) return fail(MD_EINVAL, "x and v are required");
    if (!(v->L > 0.0)) return fail(MD_EINVAL, "L must be > 0");
    if (h.c.coulomb == 1 && h.prm.r_C > 0.5 * v->L * (1.0 + 1e-12)) return fail(MD_EINVAL, "r_C exceeds L/2");
    if (v->type) {
        for (int64_t i = 0; i < h.N; ++i)
            if (v->type[i] != (i < h.Np ? 1 : 0)) return fail(MD_EINVAL, "type must list protons first");
    }
    if (v->f && !(v->L_F > 0.0)) return fail(MD_EINVAL, "L_F must be > 0 when forces are given");
    double clock[8] = {v->L, v->L_base > 0 ? v->L_base : v->L, v->t, v->t_base, v->xi_dot, (double)v->step,
                       v->f ? v->L_F : v->L, 0.0};
    CK(cudaMemcpyAsync(h.d_stage, v->x, sizeof(double) * 3 * h.N, cudaMemcpyHostToDevice, stream_));
    CK(cudaMemcpyAsync(h.d_stage + 3 * h.N, v->v, sizeof(double) * 3 * h.N, cudaMemcpyHostToDevice, stream_));
    if (v->f)
        CK(cudaMemcpyAsync(h.d_stage + 6 * h.N, v->f, sizeof(double) * 3 * h.N, cudaMemcpyHostToDevice, stream_));
    CK(cudaMemcpyAsync(d_clock_, clock, sizeof(clock), cudaMemcpyHostToDevice, stream_));
    int rc;
    if (v->f && !h.dirty) {
        // the caller's forces: the state goes into the current slot order and
        // the rebuild rule decides (a state saved from this system keeps its
        // tiles), then the forces are placed by particle id
        launch_load_sorted(H_, stream_, idx, h.d_stage, h.d_stage + 3 * h.N, v->L);
        launch_set_clock(H_, stream_, idx, d_clock_, true);
        launch_rebuild(H_, stream_, 0, idx);
        launch_scatter_forces(H_, stream_, idx, h.d_stage + 6 * h.N);
        CK(cudaGetLastError());
        h.dirty = false;
    } else if (v->f) {
        // (a system whose tiles are not current: sort into tiles from the original order)
        launch_set_clock(H_, stream_, idx, d_clock_);
        launch_scatter_state(H_, stream_, idx, h.d_stage, h.d_stage + 3 * h.N);
        launch_rebuild(H_, stream_, 1, idx);
        launch_scatter_forces(H_, stream_, idx, h.d_stage + 6 * h.N);
        CK(cudaGetLastError());
        h.dirty = false;
    } else {
        launch_set_clock(H_, stream_, idx, d_clock_);
        launch_scatter_state(H_, stream_, idx, h.d_stage, h.d_stage + 3 * h.N);
        if ((rc = refresh(idx))) return rc;
    }
    h.host_step = v->step;
    h.xi = v->xi_dot;
    return check_errors();
}

int Engine::set_params(int idx, const md_params& p) {
    SysHost& h = *sys[idx];
    const double rC = p.r_C > 0.0 ? p.r_C : std::min(40.0, 0.5 * h.L0);
    if (p.coulomb < 0 || p.coulomb > 2) return fail(MD_EINVAL, "coulomb must be 0, 1 or 2");
    if (p.coulomb == 1 && rC > 0.5 * h.L0 * (1.0 + 1e-12)) return fail(MD_EINVAL, "r_C exceeds L0/2");
    if (!(p.dt > 0.0) || !(p.r_nuc > 0.0) || !(p.skin > 0.0) || !(p.lambda_s >= 0.0))
        return fail(MD_EINVAL, "dt, r_nuc, skin must be > 0 and lambda_s >= 0");
    if (p.affine != 0 && p.affine != 1) return fail(MD_EINVAL, "affine must be 0 or 1");
    if (p.force_unroll < 0 || p.force_unroll > 4)
        return fail(MD_EINVAL, "force_unroll must be 0, 1, 2, 3 or 4");
    if (p.precision != MD_PREC_SPLIT && p.precision != MD_PREC_FP64) return fail(MD_EINVAL, "bad precision");
    if (p.sort_bits != 0 && (p.sort_bits < 2 || p.sort_bits > 7)) return fail(MD_EINVAL, "sort_bits in 2..7");
    if (p.list_kind != 0 && p.list_kind != 1) return fail(MD_EINVAL, "list_kind must be 0 or 1");
    if (p.list_kind == 1 && p.precision != MD_PREC_SPLIT)
        return fail(MD_EINVAL, "Verlet lists (list_kind 1) need split precision");
    if (p.list_kind == 1 && !(p.verlet_pool > 0.0)) return fail(MD_EINVAL, "verlet_pool must be > 0");
    if (p.uf_iter_limit < 1 || p.uf_iter_limit > 0x7fffffff)
        return fail(MD_EINVAL, "uf_iter_limit must be in [1, 2^31 - 1]");
    if (p.persistent < -1 || p.persistent > 1) return fail(MD_EINVAL, "persistent must be -1, 0 or 1");
    if (p.persistent == 1 && (p.precision == MD_PREC_FP64 || p.list_kind != 0 || p.coulomb == 2))
        return fail(MD_EINVAL, "the persistent step needs split precision, tile lists and coulomb 0 or 1");
    if (p.wait_limit_ns < 1) return fail(MD_EINVAL, "wait_limit_ns must be >= 1");
    const int nbits = p.sort_bits ? p.sort_bits : auto_bits(h.N);
    if (p.list_kind == 1) {
        // (re)allocate the list pool when it is missing or too small
        const long long cap = verlet_capacity(h.N, h.Np, h.L0, h.T, p, rC);
        if (h.c.vlist == nullptr || cap > h.c.vcap) {
            cudaStreamSynchronize(stream_);
            drop_graphs();
            void* old[] = {h.c.vlist, h.c.vcount, h.c.voff, h.c.vwidth};
            for (void* q : old)
                if (q) {
                    cudaFree(q);
                    h.allocs.erase(std::find(h.allocs.begin(), h.allocs.end(), q));
                }
            h.c.vlist = nullptr;
            h.c.vcount = nullptr;
            h.c.voff = nullptr;
            h.c.vwidth = nullptr;
            int rc = dalloc(h, &h.c.vlist, (size_t)cap);
            if (!rc) rc = dalloc(h, &h.c.vcount, (size_t)h.T * kTile);
            if (!rc) rc = dalloc(h, &h.c.voff, (size_t)h.T);
            if (!rc) rc = dalloc(h, &h.c.vwidth, (size_t)h.T);
            if (rc) return rc;
            h.c.vcap = cap;
        }
    }
    if (p.precision != precision) {
        if (sys.size() > 1) return fail(MD_EINVAL, "precision is shared by all systems of a batch");
        precision = p.precision;
        H_.precision = precision;
        cudaStreamSynchronize(stream_);
        drop_graphs();
    }
    if (idx == 0) H_.fixed_var = fixed_variant((int)p.force_unroll, H_.dev.tune_variants != 0);
    if ((h.prm.cond_graph != 0) != (p.cond_graph != 0) || h.prm.force_unroll != p.force_unroll) {   // graph layout
        cudaStreamSynchronize(stream_);
        drop_graphs();
    }
    h.prm = p;
    h.prm.r_C = rC;
    if (p.lambda_s == 0.0) h.prm.lambda_s = lambda_thomas_fermi((double)h.Np / (h.L0 * h.L0 * h.L0));
    SysConst& c = h.c;
    c.dt = p.dt;
    c.hkick = 0.5 * c.dt / c.M;
    c.dtf = (float)c.dt;
    c.T_target = p.T;
    c.skin = p.skin;
    c.lambda_s = h.prm.lambda_s;
    c.affine = p.affine;
    c.r_nuc = p.r_nuc;
    c.r_C = rC;
    c.r_pp = p.r_pp;
    c.r_np = p.r_np;
    c.relax_gamma = p.relax_gamma;
    c.relax_dmax = p.relax_dmax;
    c.thermostat_every = (int)p.thermostat_every;
    c.rebuild_every = (int)std::max<int64_t>(1, p.rebuild_every);
    const bool pp_changed = (c.coulomb == 2) != (p.coulomb == 2);
    const bool lists_changed = c.list_kind != p.list_kind;
    c.coulomb = p.coulomb;
    c.energy_every = (int)p.energy_every;
    c.list_kind = p.list_kind;
    c.force_unroll = p.force_unroll;
    c.uf_limit = (int)p.uf_iter_limit;
    c.pf = pair_consts(c);
    if (idx == 0 && (p.persistent != h.prm.persistent || p.wait_limit_ns != h.prm.wait_limit_ns)) {
        cudaStreamSynchronize(stream_);
        drop_graphs();
    }
    if (pp_changed || lists_changed) {
        cudaStreamSynchronize(stream_);
        drop_graphs();
        H_.any_pp = false;
        H_.any_verlet = false;
        for (SysHost* q : sys) {
            H_.any_pp |= (q->c.coulomb == 2);
            H_.any_verlet |= (q->c.list_kind == 1);
        }
    }
    {
        const bool was = persistent_;
        int rc = persistent_mode();
        if (rc) return rc;
        if (was != persistent_) {
            cudaStreamSynchronize(stream_);
            drop_graphs();
            long long ntot = 0;
            for (SysHost* q : sys) ntot += q->N;
            H_.dev.tune_variants = (precision != MD_PREC_FP64 && ntot >= kVariantMinN && !persistent_) ? 1 : 0;
            H_.fixed_var = fixed_variant((int)sys[0]->prm.force_unroll, H_.dev.tune_variants != 0);
        }
    }
    if (nbits != h.nbits) {
        // a different sort grid resizes the engine's bin tables
        h.nbits = nbits;
        h.nbins = 1ll << (3 * nbits);
        c.nbits = nbits;
        c.nbins = h.nbins;
        int rc = build_tables();
        if (rc) return rc;
    } else {
        CK(cudaMemcpyAsync(d_sys_ + idx, &c, sizeof(SysConst), cudaMemcpyHostToDevice, stream_));
    }
    int one = 1;
    CK(cudaMemcpyAsync(&h.d_st->force_rebuild, &one, sizeof(int), cudaMemcpyHostToDevice, stream_));
    h.dirty = true;
    CK(cudaStreamSynchronize(stream_));
    return MD_OK;
}

// Short timed trials over pair-list skin x spatial-sort resolution from a
// saved state; the fastest setting is kept and the state restored.
int Engine::autotune(int64_t steps, md_params* chosen) {
    if (steps < 1) return fail(MD_EINVAL, "steps must be >= 1");
    const int n = (int)sys.size();
    std::vector<std::vector<double>> xs(n), vs(n);
    std::vector<md_state_view> saved(n);
    std::vector<md_params> base(n);
    int rc;
    for (int s = 0; s < n; ++s) {
        xs[s].resize(3 * sys[s]->N);
        vs[s].resize(3 * sys[s]->N);
        md_state_view v{};
        v.x = xs[s].data();
        v.v = vs[s].data();
        if ((rc = get_state(s, &v))) return rc;
        saved[s] = v;
        base[s] = sys[s]->prm;
    }
    const double skins[] = {0.5, 1.0, 1.5, 2.0};
    const int dbits[] = {-1, 0, 1};
    // force-pass code variants (loop unrolling, i.e. instruction footprint):
    // tried where the step runs one fixed variant, the persistent step kernel
    // (graph steps of large engines choose theirs on the device)
    std::vector<int> codes(1, base[0].force_unroll);
    if (persistent_ && base[0].force_unroll == 0) codes = {4, 2, 1};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    double best_skin = base[0].skin;
    int best_d = 0, best_code = codes[0];
    for (int code : codes) {
        for (double sk : skins) {
            for (int d : dbits) {
                for (int s = 0; s < n; ++s) {
                    md_params p = base[s];
                    p.skin = sk;
                    p.sort_bits = std::min(7, std::max(2, auto_bits(sys[s]->N) + d));
                    p.force_unroll = code;
                    if ((rc = set_params(s, p)) || (rc = set_state(s, &saved[s]))) goto done;
                }
                if ((rc = step(2, nullptr))) goto done;
                CK(cudaEventRecord(e0, stream_));
                if ((rc = step_async(steps, nullptr, nullptr))) goto done;
                CK(cudaEventRecord(e1, stream_));
                if ((rc = check_errors())) goto done;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) {
                    best = ms;
                    best_skin = sk;
                    best_d = d;
                    best_code = code;
                }
            }
        }
    }
    for (int s = 0; s < n; ++s) {
        md_params p = base[s];
        p.skin = best_skin;
        p.sort_bits = std::min(7, std::max(2, auto_bits(sys[s]->N) + best_d));
        p.force_unroll = best_code;
        if ((rc = set_params(s, p)) || (rc = set_state(s, &saved[s]))) goto done;
        sys[s]->host_step = saved[s].step;
    }
    if (chosen) *chosen = sys[0]->prm;
    rc = MD_OK;
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

int Engine::info(int idx, md_info_t* out) {
    SysHost& h = *sys[idx];
    SysState st;
    CK(cudaMemcpyAsync(&st, h.d_st, sizeof(st), cudaMemcpyDeviceToHost, stream_));
    CK(cudaStreamSynchronize(stream_));
    out->N = h.N;
    out->Np = h.Np;
    out->tiles = h.T;
    out->rebuilds = st.n_rebuilds;
    out->list_entries = st.list_total;
    unsigned long long cond_runs = 0;
    CK(cudaMemcpyAsync(&cond_runs, d_cond_runs_, sizeof(cond_runs), cudaMemcpyDeviceToHost, stream_));
    CK(cudaStreamSynchronize(stream_));
    out->launches = launches + (int64_t)cond_runs * cond_nodes_;
    out->device_bytes = (int64_t)(h.bytes + (sys.size() == 1 ? table_bytes_ : 0));
    out->need_wrap = st.need_wrap;
    out->sort_bits = h.nbits;
    out->tile_halfext_mean = h.T ? (double)st.hsum / h.T : 0.0;
    out->tile_halfext_max = (double)__uint_as_float_host(st.hmax);
    out->verlet_entries = h.c.list_kind == 1 ? (int64_t)st.vpairs : 0;
    out->verlet_slots = h.c.list_kind == 1 ? (int64_t)st.vtop : 0;
    out->verlet_capacity = h.c.list_kind == 1 ? (int64_t)h.c.vcap : 0;
    ForceTune tu{};
    CK(cudaMemcpyAsync(&tu, d_tune_, sizeof(tu), cudaMemcpyDeviceToHost, stream_));
    CK(cudaStreamSynchronize(stream_));
    static const int code[kVariants] = {4, 2, 1, 3};
    const int fu = (int)h.prm.force_unroll;
    out->force_code = H_.dev.tune_variants ? code[tu.sel < 0 || tu.sel >= kVariants ? 0 : tu.sel] : code[fixed_variant(fu, false)];
    out->force_trials = tu.trials;
    return MD_OK;
}

}  // namespace pasta
