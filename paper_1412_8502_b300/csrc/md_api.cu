// C ABI of the nucleon MD library (declarations and contracts in md.h).
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "engine.h"

using pasta::Engine;
using pasta::fail;

namespace pasta {
const char* last_error_cstr();
}

struct md_system {
    Engine* eng;
    int idx;
    bool owner;
};

struct md_batch {
    Engine* eng;
    std::vector<md_system*> views;
    std::vector<double> xi;
};

namespace {

int check_device() {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        cudaGetLastError();
        return fail(MD_ENODEV, "no CUDA device available");
    }
    return MD_OK;
}

#define GUARD(h)                                                        \
    do {                                                                \
        if (!(h)) return fail(MD_EINVAL, "null handle");                \
    } while (0)

}  // namespace

extern "C" {

void md_params_default(md_params* p) {
    if (!p) return;
    p->dt = 2.0;
    p->r_nuc = 11.5;
    p->r_C = 0.0;
    p->lambda_s = 10.0;
    p->skin = 1.0;
    p->rebuild_every = 10;
    p->thermostat_every = 100;
    p->T = 0.0;
    p->precision = MD_PREC_SPLIT;
    p->coulomb = 1;
    p->r_pp = 4.5;
    p->r_np = 3.0;
    p->relax_iters = 500;
    p->relax_gamma = 0.002;
    p->relax_dmax = 0.1;
    p->energy_every = 0;
    p->sort_bits = 0;
    p->affine = 0;
    p->list_kind = 0;
    p->verlet_pool = 2.0;
    p->cond_graph = 1;
    p->force_unroll = 0;
    p->uf_iter_limit = 1ll << 26;
    p->wait_limit_ns = 2000000000ll;
    p->persistent = -1;
}

double md_lambda_thomas_fermi(double n_e) { return pasta::lambda_thomas_fermi(n_e); }

const char* md_last_error(void) { return pasta::last_error_cstr(); }

int md_debug_fail_alloc(int64_t nth) {
    if (nth < 0) return fail(MD_EINVAL, "nth must be >= 0");
    pasta::arm_alloc_failure((long long)nth);
    return MD_OK;
}

int md_create_ex(int64_t N, double Yp, double rho, double T, uint64_t seed, const md_params* p, md_system** out) {
    if (!out) return fail(MD_EINVAL, "out is null");
    *out = nullptr;
    int rc = check_device();
    if (rc) return rc;
    md_params prm;
    if (p) prm = *p;
    else md_params_default(&prm);
    Engine* e = new (std::nothrow) Engine();
    if (!e) return fail(MD_ENOMEM, "host allocation failed");
    if ((rc = e->add_system(N, Yp, rho, T, seed, prm)) || (rc = e->build_tables()) || (rc = e->initialise())) {
        delete e;
        return rc;
    }
    *out = new md_system{e, 0, true};
    return MD_OK;
}

int md_create(int64_t N, double Yp, double rho, double T, uint64_t seed, md_system** out) {
    return md_create_ex(N, Yp, rho, T, seed, nullptr, out);
}

int md_destroy(md_system* s) {
    if (!s) return MD_OK;
    if (!s->owner) return fail(MD_EINVAL, "system belongs to a batch");
    delete s->eng;
    delete s;
    return MD_OK;
}

int md_get_params(const md_system* s, md_params* p) {
    GUARD(s);
    if (!p) return fail(MD_EINVAL, "p is null");
    *p = s->eng->sys[s->idx]->prm;
    return MD_OK;
}

int md_set_params(md_system* s, const md_params* p) {
    GUARD(s);
    if (!p) return fail(MD_EINVAL, "p is null");
    return s->eng->set_params(s->idx, *p);
}

int md_set_stream(md_system* s, void* stream) {
    GUARD(s);
    s->eng->set_stream((cudaStream_t)stream);
    return MD_OK;
}

int md_step(md_system* s, int64_t n, double xi_dot) {
    GUARD(s);
    if (!std::isfinite(xi_dot)) return fail(MD_EINVAL, "xi_dot must be finite");
    if (!s->owner) return fail(MD_EINVAL, "step a batch member through md_batch_step");
    std::vector<double> xi(1, xi_dot);
    return s->eng->step(n, &xi);
}

int md_step_async(md_system* s, int64_t n, double xi_dot) {
    GUARD(s);
    if (!std::isfinite(xi_dot)) return fail(MD_EINVAL, "xi_dot must be finite");
    if (!s->owner) return fail(MD_EINVAL, "step a batch member through md_batch_step");
    if (n < 0) return fail(MD_EINVAL, "n must be >= 0");
    std::vector<double> xi(1, xi_dot);
    return s->eng->step_async(n, &xi, nullptr);
}

int md_sync(md_system* s) {
    GUARD(s);
    return s->eng->check_errors();
}

int md_forces(md_system* s, double* f_out) {
    GUARD(s);
    if (!f_out) return fail(MD_EINVAL, "f_out is null");
    return s->eng->forces(s->idx, f_out);
}

int md_energy(md_system* s, md_energy_t* out) {
    GUARD(s);
    if (!out) return fail(MD_EINVAL, "out is null");
    return s->eng->energy(s->idx, out);
}

int md_step_energy(md_system* s, md_energy_t* out) {
    GUARD(s);
    if (!out) return fail(MD_EINVAL, "out is null");
    return s->eng->step_energy(s->idx, out);
}

int md_clusters(md_system* s, int32_t* labels, int64_t* hist_A, int64_t* hist_Z, md_cluster_stats* st) {
    GUARD(s);
    return s->eng->clusters(s->idx, labels, hist_A, hist_Z, st);
}

int md_clusters_mste(md_system* s, int32_t* labels, int64_t* hist_A, int64_t* hist_Z, md_cluster_stats* st) {
    GUARD(s);
    return s->eng->clusters_mste(s->idx, labels, hist_A, hist_Z, st);
}

int md_get_state(md_system* s, md_state_view* v) {
    GUARD(s);
    if (!v) return fail(MD_EINVAL, "view is null");
    return s->eng->get_state(s->idx, v);
}

int md_set_state(md_system* s, const md_state_view* v) {
    GUARD(s);
    if (!v) return fail(MD_EINVAL, "view is null");
    return s->eng->set_state(s->idx, v);
}

int md_get_info(const md_system* s, md_info_t* info) {
    GUARD(s);
    if (!info) return fail(MD_EINVAL, "info is null");
    return s->eng->info(s->idx, info);
}

int md_set_timing(md_system* s, int on) {
    GUARD(s);
    if (on < 0 || on > 2) return fail(MD_EINVAL, "timing level must be 0, 1 or 2");
    s->eng->set_timing(on);
    return MD_OK;
}

int md_kernel_times(md_system* s, int max, const char** names, int64_t* launches, double* ms, int* n) {
    GUARD(s);
    return s->eng->kernel_times(max, names, launches, ms, n);
}

int md_autotune(md_system* s, int64_t steps, md_params* chosen) {
    GUARD(s);
    if (!s->owner) return fail(MD_EINVAL, "tune a batch through md_batch_autotune");
    return s->eng->autotune(steps, chosen);
}

// ------------------------------------------------------------------ batch
int md_batch_create(int n, const md_job* jobs, const md_params* p, md_batch** out) {
    if (!out || !jobs || n <= 0) return fail(MD_EINVAL, "need n > 0 jobs and an out pointer");
    *out = nullptr;
    int rc = check_device();
    if (rc) return rc;
    md_params prm;
    if (p) prm = *p;
    else md_params_default(&prm);
    Engine* e = new (std::nothrow) Engine();
    if (!e) return fail(MD_ENOMEM, "host allocation failed");
    for (int i = 0; i < n && !rc; ++i)
        rc = e->add_system(jobs[i].N, jobs[i].Yp, jobs[i].rho, jobs[i].T, jobs[i].seed, prm);
    if (!rc) rc = e->build_tables();
    if (!rc) rc = e->initialise();
    if (rc) {
        delete e;
        return rc;
    }
    md_batch* b = new md_batch();
    b->eng = e;
    for (int i = 0; i < n; ++i) {
        b->views.push_back(new md_system{e, i, false});
        b->xi.push_back(jobs[i].xi_dot);
    }
    *out = b;
    return MD_OK;
}

int md_batch_step(md_batch* b, int64_t n) {
    GUARD(b);
    return b->eng->step(n, &b->xi);
}

int md_batch_autotune(md_batch* b, int64_t steps, md_params* chosen) {
    GUARD(b);
    return b->eng->autotune(steps, chosen);
}

int md_batch_system(md_batch* b, int i, md_system** out) {
    GUARD(b);
    if (!out || i < 0 || i >= (int)b->views.size()) return fail(MD_EINVAL, "index out of range");
    *out = b->views[i];
    return MD_OK;
}

int md_batch_destroy(md_batch* b) {
    if (!b) return MD_OK;
    for (md_system* v : b->views) delete v;
    delete b->eng;
    delete b;
    return MD_OK;
}

}  // extern "C"
