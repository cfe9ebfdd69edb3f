// capi.cu -- C ABI of the GB300 N-body/SPH library (declared in galnb.h).
//
// The calls follow the problem statement of Hirashima et al. (SC'25, arXiv
// 2510.23330): particles with FP64 positions, FP32 velocity, mass and
// per-particle softening (Sec. 3.5, 4.3); tree build (Sec. 3.4); gravity,
// SPH density and force (Table 3); shared-timestep leapfrog (Sec. 3.2).
// All device work runs on cfg.cuda_stream; each call ends with one stream
// synchronisation and a check of the device status word.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace gnb {

int fail(gnb_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    return code;
}

int cuda_check(gnb_ctx *c, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return GNB_OK;
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(c, GNB_ENOMEM, m);
    return fail(c, GNB_ECUDA, m);
}

void dfree(gnb_ctx *, void *p)
{
    if (p) cudaFree(p);
}

static void parr_free(gnb_ctx *c, PArr &p)
{
    void *all[] = {p.x, p.y, p.z, p.h2, p.id, p.vx, p.vy, p.vz, p.m, p.eps, p.u, p.rx, p.ry, p.rz,
                   p.vpx, p.vpy, p.vpz, p.up, p.orig, p.grank, p.cx, p.cy, p.cz, p.type};
    for (void *q : all) dfree(c, q);
    p = PArr();
}

static int parr_alloc(gnb_ctx *c, PArr &p, size_t n)
{
    GNB_TRY(dalloc(c, &p.x, n)); GNB_TRY(dalloc(c, &p.y, n)); GNB_TRY(dalloc(c, &p.z, n));
    GNB_TRY(dalloc(c, &p.h2, n)); GNB_TRY(dalloc(c, &p.id, n));
    GNB_TRY(dalloc(c, &p.vx, n)); GNB_TRY(dalloc(c, &p.vy, n)); GNB_TRY(dalloc(c, &p.vz, n));
    GNB_TRY(dalloc(c, &p.m, n)); GNB_TRY(dalloc(c, &p.eps, n)); GNB_TRY(dalloc(c, &p.u, n));
    GNB_TRY(dalloc(c, &p.rx, n)); GNB_TRY(dalloc(c, &p.ry, n)); GNB_TRY(dalloc(c, &p.rz, n));
    GNB_TRY(dalloc(c, &p.vpx, n)); GNB_TRY(dalloc(c, &p.vpy, n)); GNB_TRY(dalloc(c, &p.vpz, n));
    GNB_TRY(dalloc(c, &p.up, n));
    GNB_TRY(dalloc(c, &p.orig, n)); GNB_TRY(dalloc(c, &p.grank, n));
    GNB_TRY(dalloc(c, &p.cx, n)); GNB_TRY(dalloc(c, &p.cy, n)); GNB_TRY(dalloc(c, &p.cz, n));
    GNB_TRY(dalloc(c, &p.type, n));
    return GNB_OK;
}

static void free_particles(gnb_ctx *c)
{
    parr_free(c, c->P[0]);
    parr_free(c, c->P[1]);
    void *all[] = {c->ax, c->ay, c->az, c->pot, c->dudt, c->gax, c->gay, c->gaz, c->pext, c->rho, c->pres,
                   c->cs, c->kres, c->skey, c->skey2, c->sval, c->sval2, c->slot_of_orig, c->src, c->rs_counts,
                   c->gas_flag, c->pscan, c->tmp_out};
    for (void *q : all) dfree(c, q);
    c->ax = c->ay = c->az = c->pot = c->dudt = c->gax = c->gay = c->gaz = c->pext = nullptr;
    c->rho = c->pres = c->cs = nullptr;
    c->kres = nullptr;
    c->skey = c->skey2 = nullptr;
    c->sval = c->sval2 = c->slot_of_orig = c->src = c->rs_counts = c->gas_flag = c->pscan = nullptr;
    c->tmp_out = nullptr;
    tree_free(c, c->t);
    c->cap = 0;
}

static void free_gas(gnb_ctx *c)
{
    void *all[] = {c->gslot, c->gkey, c->gcx, c->gcy, c->gcz, c->ggrank, c->grx, c->gry, c->grz, c->gx, c->gy,
                   c->gz, c->gm, c->gvx, c->gvy, c->gvz, c->gu, c->gh2, c->gh, c->g64, c->grho, c->gP, c->gcs,
                   c->gRprev, c->gE, c->nbr, c->nd2, c->mut, c->rcnt, c->roff, c->rfill, c->rlist, c->hax,
                   c->hay, c->haz, c->hdu, c->kflag, c->kR, c->kRb, c->kitem, c->gvsig, c->kwl[0], c->kwl[1],
                   c->gh2lo, c->gh2hi, c->fC, c->fR, c->fV, c->fQ};
    for (void *q : all) dfree(c, q);
    c->gslot = nullptr; c->gkey = nullptr; c->gcx = c->gcy = c->gcz = c->ggrank = nullptr;
    c->grx = c->gry = c->grz = nullptr; c->gx = c->gy = c->gz = nullptr;
    c->gm = c->gvx = c->gvy = c->gvz = c->gu = nullptr; c->gh2 = nullptr; c->gh = nullptr; c->g64 = nullptr;
    c->grho = c->gP = c->gcs = c->gRprev = c->gE = nullptr; c->nbr = nullptr; c->nd2 = nullptr; c->mut = nullptr;
    c->rcnt = c->roff = c->rfill = c->rlist = nullptr; c->hax = c->hay = c->haz = c->hdu = nullptr;
    c->kflag = nullptr; c->kR = nullptr; c->kRb = nullptr; c->kitem = nullptr; c->gvsig = nullptr;
    c->kwl[0] = c->kwl[1] = nullptr;
    c->gh2lo = c->gh2hi = nullptr;
    c->fC = nullptr; c->fR = nullptr; c->fV = nullptr; c->fQ = nullptr;
    tree_free(c, c->gt);
    c->gcap = 0;
}

static int alloc_particles(gnb_ctx *c, int64_t n)
{
    if (c->cap >= n) return GNB_OK;
    free_particles(c);
    size_t N = (size_t)n;
    GNB_TRY(parr_alloc(c, c->P[0], N));
    GNB_TRY(parr_alloc(c, c->P[1], N));
    GNB_TRY(dalloc(c, &c->ax, N)); GNB_TRY(dalloc(c, &c->ay, N)); GNB_TRY(dalloc(c, &c->az, N));
    GNB_TRY(dalloc(c, &c->pot, N)); GNB_TRY(dalloc(c, &c->dudt, N));
    GNB_TRY(dalloc(c, &c->gax, N)); GNB_TRY(dalloc(c, &c->gay, N)); GNB_TRY(dalloc(c, &c->gaz, N));
    GNB_TRY(dalloc(c, &c->pext, N)); GNB_TRY(dalloc(c, &c->rho, N)); GNB_TRY(dalloc(c, &c->pres, N));
    GNB_TRY(dalloc(c, &c->cs, N));
    GNB_TRY(dalloc(c, &c->kres, 3 * N)); GNB_TRY(dalloc(c, &c->skey, N)); GNB_TRY(dalloc(c, &c->skey2, N));
    GNB_TRY(dalloc(c, &c->sval, N)); GNB_TRY(dalloc(c, &c->sval2, N));
    GNB_TRY(dalloc(c, &c->slot_of_orig, N)); GNB_TRY(dalloc(c, &c->src, N));
    GNB_TRY(dalloc(c, &c->gas_flag, N + 1)); GNB_TRY(dalloc(c, &c->pscan, N + 1));
    GNB_TRY(dalloc(c, &c->tmp_out, 8 * N + 64));
    int ntiles = (int)((n + 2047) / 2048);
    GNB_TRY(dalloc(c, &c->rs_counts, (size_t)ntiles * 256));
    c->cap = n;
    return GNB_OK;
}

static int alloc_gas(gnb_ctx *c, int64_t ng)
{
    if (c->gcap >= ng && c->gslot) return GNB_OK;
    free_gas(c);
    size_t G = (size_t)(ng > 0 ? ng : 1);
    GNB_TRY(dalloc(c, &c->gslot, G)); GNB_TRY(dalloc(c, &c->gkey, G));
    GNB_TRY(dalloc(c, &c->gcx, G)); GNB_TRY(dalloc(c, &c->gcy, G)); GNB_TRY(dalloc(c, &c->gcz, G));
    GNB_TRY(dalloc(c, &c->ggrank, G));
    GNB_TRY(dalloc(c, &c->grx, G)); GNB_TRY(dalloc(c, &c->gry, G)); GNB_TRY(dalloc(c, &c->grz, G));
    GNB_TRY(dalloc(c, &c->gx, G)); GNB_TRY(dalloc(c, &c->gy, G)); GNB_TRY(dalloc(c, &c->gz, G));
    GNB_TRY(dalloc(c, &c->gm, G)); GNB_TRY(dalloc(c, &c->gvx, G)); GNB_TRY(dalloc(c, &c->gvy, G));
    GNB_TRY(dalloc(c, &c->gvz, G)); GNB_TRY(dalloc(c, &c->gu, G));
    GNB_TRY(dalloc(c, &c->gh2, G)); GNB_TRY(dalloc(c, &c->gh, G)); GNB_TRY(dalloc(c, &c->g64, G));
    GNB_TRY(dalloc(c, &c->grho, G)); GNB_TRY(dalloc(c, &c->gP, G)); GNB_TRY(dalloc(c, &c->gcs, G));
    GNB_TRY(dalloc(c, &c->gRprev, G)); GNB_TRY(dalloc(c, &c->gE, G)); GNB_TRY(dalloc(c, &c->gvsig, G));
    GNB_TRY(dalloc(c, &c->nbr, G * 64)); GNB_TRY(dalloc(c, &c->nd2, G * 64)); GNB_TRY(dalloc(c, &c->mut, G));
    GNB_TRY(dalloc(c, &c->rcnt, G + 1)); GNB_TRY(dalloc(c, &c->roff, G + 1)); GNB_TRY(dalloc(c, &c->rfill, G + 1));
    GNB_TRY(dalloc(c, &c->rlist, G * 64));
    cudaMemsetAsync(c->nbr, 0, sizeof(int) * G * 64, c->s);  // list entries are always valid indices
    GNB_TRY(dalloc(c, &c->hax, G)); GNB_TRY(dalloc(c, &c->hay, G)); GNB_TRY(dalloc(c, &c->haz, G));
    GNB_TRY(dalloc(c, &c->hdu, G));
    GNB_TRY(dalloc(c, &c->kflag, 2 * G + 1)); GNB_TRY(dalloc(c, &c->kR, 2 * G + 1));
    GNB_TRY(dalloc(c, &c->kRb, 2 * G + 1)); GNB_TRY(dalloc(c, &c->kitem, 2 * G + 1));
    GNB_TRY(dalloc(c, &c->kwl[0], 2 * G + 1)); GNB_TRY(dalloc(c, &c->kwl[1], 2 * G + 1));
    GNB_TRY(dalloc(c, &c->gh2lo, G)); GNB_TRY(dalloc(c, &c->gh2hi, G));
    GNB_TRY(dalloc(c, &c->fC, G)); GNB_TRY(dalloc(c, &c->fR, G)); GNB_TRY(dalloc(c, &c->fV, G));
    GNB_TRY(dalloc(c, &c->fQ, G));
    c->gcap = ng;
    return GNB_OK;
}

// After a synchronisation: translate and clear the device status word.
static int check_status(gnb_ctx *c)
{
    GNB_TRY(cuda_check(c, cudaStreamSynchronize(c->s), "stream synchronize"));
    GNB_TRY(cuda_check(c, cudaGetLastError(), "kernel"));
    int st = 0;
    GNB_TRY(cuda_check(c, cudaMemcpy(&st, c->status_d, sizeof(int), cudaMemcpyDeviceToHost), "status read"));
    if (st == 0) return GNB_OK;
    cudaMemsetAsync(c->status_d, 0, sizeof(int), c->s);
    if (st & ST_BAD_INPUT) return fail(c, GNB_EINVAL, "non-finite particle position");
    if (st & ST_TREE_OVERFLOW) return fail(c, GNB_ECAPACITY, "tree node capacity exceeded");
    if (st & ST_STACK_OVERFLOW) return fail(c, GNB_ECAPACITY, "tree walk stack overflow");
    if (st & ST_KNN_OVERFLOW) return fail(c, GNB_ECAPACITY, "kNN selection buffer overflow");
    return fail(c, GNB_ECAPACITY, "device status " + std::to_string(st));
}

// ---------------------------------------------------------------- kernels used by set_particles
__global__ void k_set_init(PArr p, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    p.orig[i] = i;
    p.h2[i] = 0.0;
    p.vpx[i] = p.vx[i]; p.vpy[i] = p.vy[i]; p.vpz[i] = p.vz[i];
    if (p.type[i] != GNB_GAS) p.u[i] = 0.f;
    p.up[i] = p.u[i];
}

__global__ void k_validate(PArr p, int n, int *bad)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int b = 0;
    if (!isfinite(p.x[i]) || !isfinite(p.y[i]) || !isfinite(p.z[i])) b |= 1;
    if (p.type[i] > 1) b |= 2;
    if (!(p.m[i] > 0.f) || !isfinite(p.m[i])) b |= 4;
    if (!(p.eps[i] >= 0.f) || !isfinite(p.eps[i])) b |= 8;
    if (p.eps[i] == 0.f) b |= 16;
    if (p.eps[i] != p.eps[0]) b |= 32;
    if (b) atomicOr(bad, b);
}

__global__ void k_gas_flag_in(const uint8_t *__restrict__ type, int *__restrict__ flag, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = type[i] == GNB_GAS;
}

__global__ void k_grank(const uint8_t *__restrict__ type, const int *__restrict__ off, int n, int *__restrict__ grank)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) grank[i] = type[i] == GNB_GAS ? off[i] : -1;
}

}  // namespace gnb

using namespace gnb;

extern "C" {

void gnb_config_default(gnb_config *cfg)
{
    if (!cfg) return;
    cfg->G = 1.0;
    cfg->theta = 0.5;
    cfg->gamma = 5.0 / 3.0;
    cfg->alpha_visc = 1.0;
    cfg->n_leaf = 16;
    cfg->n_group = 64;
    cfg->n_ngb = 64;
    cfg->multipole = 1;
    cfg->nfw_ms = 0.0;
    cfg->nfw_rs = 8.0;
    cfg->cuda_stream = nullptr;
    cfg->sph_variant = 0;
}

static bool config_ok(const gnb_config *cfg)
{
    return cfg->theta >= 0.0 && cfg->G > 0.0 && cfg->n_leaf >= 1 && cfg->n_leaf <= 255 && cfg->n_group >= 1 &&
           cfg->n_ngb == 64 && cfg->gamma > 1.0 && cfg->alpha_visc >= 0.0 && cfg->nfw_ms >= 0.0 &&
           !(cfg->nfw_ms > 0.0 && !(cfg->nfw_rs > 0.0)) && (cfg->sph_variant == 0 || cfg->sph_variant == 1);
}

int gnb_set_config(gnb_ctx *c, const gnb_config *cfg)
{
    if (!c || !cfg) return GNB_EINVAL;
    if (!config_ok(cfg)) return fail(c, GNB_EINVAL, "invalid configuration");
    cudaStreamSynchronize(c->s);
    c->cfg = *cfg;
    c->s = (cudaStream_t)cfg->cuda_stream;
    c->sorted_valid = c->tree_valid = c->gravity_valid = c->density_valid = c->force_valid = c->sphf_valid = false;
    return GNB_OK;
}

int gnb_create(gnb_ctx **out, const gnb_config *cfg)
{
    if (!out || !cfg) return GNB_EINVAL;
    *out = nullptr;
    if (!config_ok(cfg)) return GNB_EINVAL;
    gnb_ctx *c = new (std::nothrow) gnb_ctx();
    if (!c) return GNB_ENOMEM;
    c->cfg = *cfg;
    c->s = (cudaStream_t)cfg->cuda_stream;
    int rc = GNB_OK;
    if ((rc = dalloc(c, &c->status_d, 4)) || (rc = dalloc(c, &c->n_d, 4)) || (rc = dalloc(c, &c->ngas_d, 4)) ||
        (rc = dalloc(c, &c->counters_d, 8)) || (rc = dalloc(c, &c->work_d, 8)) || (rc = dalloc(c, &c->box_d, 8)) ||
        (rc = dalloc(c, &c->mm_d, 8)) || (rc = dalloc(c, &c->red_d, 256 * 10 + 16)) ||
        (rc = dalloc(c, &c->rs_total, 256)) || (rc = dalloc(c, &c->rtot_d, 4)) ||
        (rc = dalloc(c, &c->scan_part, 1100)) || (rc = dalloc(c, &c->scan_poff, 1100))) {
        gnb_destroy(c);
        return rc;
    }
    if (cudaMallocHost((void **)&c->pinned_i, 64 * sizeof(int)) != cudaSuccess) {
        gnb_destroy(c);
        return GNB_ENOMEM;
    }
    // cleared on the context's stream, which may be a non-blocking one
    if (cudaMemsetAsync(c->status_d, 0, 4 * sizeof(int), c->s) != cudaSuccess ||
        cudaMemsetAsync(c->counters_d, 0, 8 * sizeof(unsigned long long), c->s) != cudaSuccess ||
        cudaStreamSynchronize(c->s) != cudaSuccess) {
        cudaGetLastError();
        gnb_destroy(c);
        return GNB_ECUDA;
    }
    *out = c;
    return GNB_OK;
}

void gnb_destroy(gnb_ctx *c)
{
    if (!c) return;
    if (c->s) cudaStreamSynchronize(c->s);
    else cudaDeviceSynchronize();
    free_particles(c);
    free_gas(c);
    hier_free(c);
    replace_free(c);
    void *all[] = {c->status_d, c->n_d, c->ngas_d, c->counters_d, c->work_d, c->box_d, c->mm_d, c->red_d,
                   c->rs_total, c->rtot_d, c->scan_part, c->scan_poff, c->gl_pool, c->gl_next, c->gl_cnt,
                   c->gl_top, c->gl_head, c->gl_ref, c->gl_lcum};
    for (void *q : all) dfree(c, q);
    if (c->pinned_i) cudaFreeHost(c->pinned_i);
    {
        void *sur[] = {c->sreg, c->rcount, c->vacc, c->vout, c->vw,  c->vcdf, c->cent_d, c->seed_d,
                       c->rsx,  c->rsi,    c->centf, c->vpa, c->vpb, c->vpc,  c->vbox, c->vcdf32, c->vcdfc};
        for (void *q : sur) dfree(c, q);
        if (c->sn_graph) cudaGraphExecDestroy(c->sn_graph);
        if (c->sna_st) {
            cudaStreamSynchronize(c->sna_st);  // a pending batch's work ends before its buffers go
            cudaStreamDestroy(c->sna_st);
        }
        if (c->sna_ev_snap) cudaEventDestroy(c->sna_ev_snap);
        if (c->sna_ev_done) cudaEventDestroy(c->sna_ev_done);
        void *sna[] = {c->sna_x, c->sna_y, c->sna_z, c->sna_h2, c->sna_m, c->sna_u, c->sna_vx, c->sna_vy, c->sna_vz,
                       c->sna_rho, c->sna_reg, c->sna_orig, c->sna_pos, c->sna_inv, c->sna_id, c->sna_seed};
        for (void *q : sna) dfree(c, q);
        for (cudaStream_t st : c->sn_st)
            if (st) cudaStreamDestroy(st);
        for (auto &row : c->sn_ev)
            for (cudaEvent_t e : row)
                if (e) cudaEventDestroy(e);
    }
    for (auto &q : c->pend) { cudaEventDestroy(q.second.first); cudaEventDestroy(q.second.second); }
    for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
    if (c->open_ev) cudaEventDestroy(c->open_ev);
    delete c;
}

int gnb_set_particles(gnb_ctx *c, int64_t n, const int64_t *id, const uint8_t *type, const double *x,
                      const double *y, const double *z, const float *vx, const float *vy, const float *vz,
                      const float *m, const float *eps, const float *u, int on_device)
{
    if (!c) return GNB_EINVAL;
    c->err.clear();
    if (n < 1 || n > (1ll << 30)) return fail(c, GNB_EINVAL, "particle count out of range");
    if (c->sna_pending) return fail(c, GNB_ESTATE, "an asynchronous surrogate batch is pending");
    if (!id || !type || !x || !y || !z || !vx || !vy || !vz || !m || !eps || !u)
        return fail(c, GNB_EINVAL, "null array");
    c->have_particles = c->sorted_valid = c->tree_valid = c->gravity_valid = c->density_valid = c->force_valid = false;
    c->sphf_valid = false;
    c->have_h = false;
    c->hier_on = c->hier_valid = false;
    c->rid_valid = false;
    GNB_TRY(alloc_particles(c, n));
    c->cur = 0;
    PArr &p = c->P[0];
    cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    size_t N = (size_t)n;
    struct { void *d; const void *s; size_t b; } cp[] = {
        {p.id, id, 8 * N}, {p.type, type, N}, {p.x, x, 8 * N}, {p.y, y, 8 * N}, {p.z, z, 8 * N},
        {p.vx, vx, 4 * N}, {p.vy, vy, 4 * N}, {p.vz, vz, 4 * N}, {p.m, m, 4 * N}, {p.eps, eps, 4 * N},
        {p.u, u, 4 * N}};
    for (auto &q : cp) GNB_TRY(cuda_check(c, cudaMemcpyAsync(q.d, q.s, q.b, k, c->s), "particle copy"));
    int ni = (int)n;
    int nb = (ni + 255) / 256;
    c->pinned_i[0] = ni;
    cudaMemcpyAsync(c->n_d, c->pinned_i, sizeof(int), cudaMemcpyHostToDevice, c->s);
    cudaMemsetAsync(c->work_d, 0, sizeof(int), c->s);
    gnb::counted(k_validate)<<<nb, 256, 0, c->s>>>(p, ni, c->work_d);
    gnb::counted(k_set_init)<<<nb, 256, 0, c->s>>>(p, ni);
    gnb::counted(k_gas_flag_in)<<<nb, 256, 0, c->s>>>(p.type, c->gas_flag, ni);
    GNB_TRY(device_scan(c, c->gas_flag, c->pscan, c->n_d, ni, c->ngas_d));
    gnb::counted(k_grank)<<<nb, 256, 0, c->s>>>(p.type, c->pscan, ni, p.grank);
    GNB_LAUNCH_CHECK(c, "set particles");
    cudaMemcpyAsync(c->pinned_i + 1, c->work_d, sizeof(int), cudaMemcpyDeviceToHost, c->s);
    cudaMemcpyAsync(c->pinned_i + 2, c->ngas_d, sizeof(int), cudaMemcpyDeviceToHost, c->s);
    cudaMemcpyAsync(c->pinned_i + 3, p.eps, sizeof(float), cudaMemcpyDeviceToHost, c->s);
    GNB_TRY(cuda_check(c, cudaStreamSynchronize(c->s), "set particles sync"));
    int bad = c->pinned_i[1];
    int ng = c->pinned_i[2];
    if (bad & 1) return fail(c, GNB_EINVAL, "non-finite position");
    if (bad & 2) return fail(c, GNB_EINVAL, "particle type not in {0, 1}");
    if (bad & 4) return fail(c, GNB_EINVAL, "mass must be positive and finite");
    if (bad & 8) return fail(c, GNB_EINVAL, "softening must be non-negative and finite");
    if (ng > 0 && ng < c->cfg.n_ngb) return fail(c, GNB_EINVAL, "fewer gas particles than SPH neighbours");
    c->min_eps_zero = (bad & 16) != 0;
    c->slots_caller = true;
    memcpy(&c->eps0, c->pinned_i + 3, sizeof(float));
    c->eps_uniform = !(bad & (16 | 32));
    c->n = n;
    c->n_gas = ng;
    GNB_TRY(alloc_gas(c, ng));
    c->stats[GNB_S_N] = n;
    c->stats[GNB_S_NGAS] = ng;
    c->have_particles = true;
    return GNB_OK;
}

int gnb_set_state(gnb_ctx *c, int64_t n, const int64_t *id, const uint8_t *type, const double *x, const double *y,
                  const double *z, const float *vx, const float *vy, const float *vz, const float *m, const float *eps,
                  const float *u, const double *h2, const float *ax, const float *ay, const float *az,
                  const float *dudt, int grav_mode, int on_device)
{
    if (!c) return GNB_EINVAL;
    c->err.clear();
    if (!ax || !ay || !az || !dudt) return fail(c, GNB_EINVAL, "null acceleration or du/dt array");
    if (grav_mode != GNB_GRAV_DIRECT && grav_mode != GNB_GRAV_TREE && grav_mode != GNB_GRAV_NONE)
        return fail(c, GNB_EINVAL, "gravity mode");
    const int rc = gnb_set_particles(c, n, id, type, x, y, z, vx, vy, vz, m, eps, u, on_device);
    if (rc != GNB_OK) return rc;
    // right after gnb_set_particles the slots are in caller order
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const size_t N = (size_t)n;
    if (h2) GNB_TRY(cuda_check(c, cudaMemcpyAsync(c->P[c->cur].h2, h2, 8 * N, k, c->s), "state copy"));
    struct { float *d; const float *s; } cp[] = {{c->ax, ax}, {c->ay, ay}, {c->az, az}, {c->dudt, dudt}};
    for (auto &q : cp) GNB_TRY(cuda_check(c, cudaMemcpyAsync(q.d, q.s, 4 * N, k, c->s), "state copy"));
    GNB_TRY(cuda_check(c, cudaStreamSynchronize(c->s), "state copy sync"));
    c->have_h = h2 != nullptr;
    c->force_valid = true;
    c->last_grav_mode = grav_mode;
    return GNB_OK;
}

}  // extern "C"

namespace gnb {

std::atomic<long long> g_launches{0};

static bool mode_ok(int mode)
{
    return mode == GNB_GRAV_DIRECT || mode == GNB_GRAV_TREE || mode == GNB_GRAV_NONE;
}

static cudaEvent_t ev_get(gnb_ctx *c)
{
    if (!c->evpool.empty()) {
        cudaEvent_t e = c->evpool.back();
        c->evpool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

void phase_begin(gnb_ctx *c, int phase)
{
    if (!c->timing) return;
    phase_end(c);
    c->open_ev = ev_get(c);
    c->open_phase = phase;
    if (c->open_ev) cudaEventRecord(c->open_ev, c->s);
}

void phase_end(gnb_ctx *c)
{
    if (!c->timing || c->open_phase < 0) return;
    cudaEvent_t e = ev_get(c);
    if (c->open_ev && e) {
        cudaEventRecord(e, c->s);
        c->pend.push_back({c->open_phase, {c->open_ev, e}});
    }
    c->open_phase = -1;
    c->open_ev = nullptr;
}

// after the stream is idle: add the recorded phase durations
static void phase_resolve(gnb_ctx *c)
{
    phase_end(c);
    for (auto &q : c->pend) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, q.second.first, q.second.second) == cudaSuccess) {
            c->phase_ms[q.first] += ms;
            c->phase_calls[q.first] += 1;
        } else {
            cudaGetLastError();
        }
        c->evpool.push_back(q.second.first);
        c->evpool.push_back(q.second.second);
    }
    c->pend.clear();
}

// Root box, keys and the Morton-order permutation of all particle arrays.
static int do_sort(gnb_ctx *c)
{
    phase_begin(c, GNB_T_SORT);
    GNB_TRY(morton_and_sort(c));
    phase_end(c);
    c->sorted_valid = true;
    c->tree_valid = false;
    return GNB_OK;
}

static int do_build(gnb_ctx *c)
{
    GNB_TRY(do_sort(c));
    phase_begin(c, GNB_T_TREE);
    PArr &a = c->P[c->cur];
    GNB_TRY(build_tree(c, c->t, c->skey, (int)c->n, c->n_d, c->cfg.n_leaf, c->cfg.n_group, a.cx, a.cy, a.cz, a.rx,
                       a.ry, a.rz, a.m, a.eps, true));
    phase_end(c);
    c->tree_valid = true;
    c->stats[GNB_S_NODES] = c->t.nnodes;
    return GNB_OK;
}

static int read_groups(gnb_ctx *c)
{
    if (!c->tree_valid) return GNB_OK;  // no gravity tree for the current positions (gravity off)
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(c->pinned_i + 8, c->t.ngroups_d, sizeof(int), cudaMemcpyDeviceToHost, c->s),
                       "groups count"));
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(c->pinned_i + 9, c->t.lvl, sizeof(int) * (GNB_MAXLEV + 2),
                                          cudaMemcpyDeviceToHost, c->s), "levels"));
    GNB_TRY(cuda_check(c, cudaStreamSynchronize(c->s), "groups sync"));
    c->t.ngroups = c->pinned_i[8];
    c->stats[GNB_S_GROUPS] = c->t.ngroups;
    int maxlev = 0;
    for (int l = 0; l <= GNB_MAXLEV; l++)
        if (c->pinned_i[9 + l + 1] > c->pinned_i[9 + l]) maxlev = l;
    c->stats[GNB_S_MAXLEVEL] = maxlev;
    return GNB_OK;
}

static int do_gravity(gnb_ctx *c, int mode)
{
    cudaMemsetAsync(c->counters_d, 0, 2 * sizeof(unsigned long long), c->s);
    phase_begin(c, GNB_T_GRAVITY);
    if (mode == GNB_GRAV_TREE) {
        GNB_TRY(gravity_tree(c));
    } else if (mode == GNB_GRAV_DIRECT) {
        GNB_TRY(gravity_direct(c));
    } else {  // GNB_GRAV_NONE: no self-gravity
        size_t b = sizeof(float) * (size_t)c->n;
        cudaMemsetAsync(c->gax, 0, b, c->s); cudaMemsetAsync(c->gay, 0, b, c->s);
        cudaMemsetAsync(c->gaz, 0, b, c->s); cudaMemsetAsync(c->pot, 0, b, c->s);
    }
    phase_begin(c, GNB_T_EXTERNAL);
    GNB_TRY(gravity_nfw(c));
    GNB_TRY(zero_forces(c));
    phase_end(c);
    c->gravity_valid = true;
    c->last_grav_mode = mode;
    return GNB_OK;
}

static int do_forces(gnb_ctx *c, int mode)
{
    // without self-gravity only the hydro tree is needed, which the sorted
    // gas particles give
    GNB_TRY(mode == GNB_GRAV_NONE ? do_sort(c) : do_build(c));
    GNB_TRY(do_gravity(c, mode));
    GNB_TRY(sph_density(c));
    c->density_valid = true;
    GNB_TRY(sph_force(c));
    c->force_valid = true;
    c->sphf_valid = true;
    return GNB_OK;
}

// One kick-drift-kick step; forces at the start of the step must be current.
static int kdk_one(gnb_ctx *c, double dt, int mode)
{
    float hdt = (float)(0.5 * dt);
    phase_begin(c, GNB_T_KDK);
    int rc = kick_drift_predict(c, hdt, dt);
    phase_end(c);
    c->sorted_valid = c->tree_valid = c->gravity_valid = c->density_valid = c->force_valid = c->sphf_valid = false;
    c->use_pred = true;
    if (rc == GNB_OK) rc = do_forces(c, mode);
    c->use_pred = false;
    phase_begin(c, GNB_T_KDK);
    if (rc == GNB_OK) rc = kick(c, hdt, true);
    phase_end(c);
    return rc;
}

static int finish(gnb_ctx *c, int rc)
{
    if (rc != GNB_OK) {
        cudaStreamSynchronize(c->s);
        cudaGetLastError();
        cudaMemsetAsync(c->status_d, 0, sizeof(int), c->s);
        phase_resolve(c);
        return rc;
    }
    rc = check_status(c);
    phase_resolve(c);
    return rc;
}

}  // namespace gnb

extern "C" {

int gnb_build_tree(gnb_ctx *c)
{
    if (!c) return GNB_EINVAL;
    c->err.clear();
    if (!c->have_particles) return fail(c, GNB_ESTATE, "no particles");
    int rc = do_build(c);
    if (rc == GNB_OK) rc = read_groups(c);
    c->gravity_valid = c->density_valid = c->force_valid = c->sphf_valid = false;
    return finish(c, rc);
}

int gnb_compute_gravity(gnb_ctx *c, int mode)
{
    if (!c) return GNB_EINVAL;
    c->err.clear();
    if (!mode_ok(mode)) return fail(c, GNB_EINVAL, "gravity mode");
    if (!c->have_particles) return fail(c, GNB_ESTATE, "no particles");
    int rc = GNB_OK;
    if (!c->tree_valid) rc = do_build(c);
    if (rc == GNB_OK) rc = do_gravity(c, mode);
    if (rc == GNB_OK) rc = read_groups(c);
    c->force_valid = false;
    return finish(c, rc);
}

int gnb_compute_sph_density(gnb_ctx *c)
{
    if (!c) return GNB_EINVAL;
    c->err.clear();
    if (!c->have_particles) return fail(c, GNB_ESTATE, "no particles");
    int rc = GNB_OK;
    if (!c->tree_valid) rc = do_build(c);
    if (rc == GNB_OK) rc = sph_density(c);
    if (rc == GNB_OK) c->density_valid = true;
    c->force_valid = false;
    return finish(c, rc);
}

int gnb_compute_sph_force(gnb_ctx *c)
{
    if (!c) return GNB_EINVAL;
    c->err.clear();
    if (!c->density_valid) return fail(c, GNB_ESTATE, "SPH density not computed for the current positions");
    int rc = GNB_OK;
    if (!c->gravity_valid) {
        size_t b = sizeof(float) * (size_t)c->n;
        cudaMemsetAsync(c->ax, 0, b, c->s); cudaMemsetAsync(c->ay, 0, b, c->s); cudaMemsetAsync(c->az, 0, b, c->s);
        cudaMemsetAsync(c->dudt, 0, b, c->s);
    }
    rc = sph_force(c);
    if (rc == GNB_OK) { c->force_valid = c->gravity_valid; c->sphf_valid = true; }
    return finish(c, rc);
}

int gnb_compute_forces(gnb_ctx *c, int mode)
{
    if (!c) return GNB_EINVAL;
    c->err.clear();
    if (!mode_ok(mode)) return fail(c, GNB_EINVAL, "gravity mode");
    if (!c->have_particles) return fail(c, GNB_ESTATE, "no particles");
    int rc = do_forces(c, mode);
    if (rc == GNB_OK) rc = read_groups(c);
    return finish(c, rc);
}

int gnb_step_kdk(gnb_ctx *c, double dt, int nsteps, int mode)
{
    if (!c) return GNB_EINVAL;
    c->err.clear();
    if (!std::isfinite(dt) || nsteps < 0) return fail(c, GNB_EINVAL, "dt or nsteps");
    if (!mode_ok(mode)) return fail(c, GNB_EINVAL, "gravity mode");
    if (!c->have_particles) return fail(c, GNB_ESTATE, "no particles");
    int rc = GNB_OK;
    if (!c->force_valid || c->last_grav_mode != mode) {
        rc = do_forces(c, mode);
        if (rc != GNB_OK) return finish(c, rc);
    }
    for (int s = 0; s < nsteps && rc == GNB_OK; s++) rc = kdk_one(c, dt, mode);
    if (rc == GNB_OK) rc = read_groups(c);
    return finish(c, rc);
}

int gnb_inject_energy(gnb_ctx *c, const double pos[3], double energy, double info[4])
{
    if (!c) return GNB_EINVAL;
    c->err.clear();
    if (!pos || !std::isfinite(pos[0]) || !std::isfinite(pos[1]) || !std::isfinite(pos[2]) ||
        !std::isfinite(energy) || energy < 0.0)
        return fail(c, GNB_EINVAL, "position or energy");
    if (!c->have_particles) return fail(c, GNB_ESTATE, "no particles");
    if (c->n_gas < c->cfg.n_ngb) return fail(c, GNB_ESTATE, "fewer gas particles than neighbours");
    double out[4] = {0, 0, 0, 0};
    int rc = inject_energy(c, pos, energy, out);
    if (info) for (int k = 0; k < 4; k++) info[k] = out[k];
    // pressure and forces depend on u
    c->density_valid = c->force_valid = c->sphf_valid = false;
    return finish(c, rc);
}

int gnb_cfl_timestep(gnb_ctx *c, double courant, double *dt)
{
    if (!c || !dt) return GNB_EINVAL;
    c->err.clear();
    if (!(courant > 0.0)) return fail(c, GNB_EINVAL, "courant factor");
    if (!c->sphf_valid) return fail(c, GNB_ESTATE, "SPH force not computed");
    double m = 0.0;
    int rc = cfl_min_h_over_vsig(c, &m);
    *dt = courant * m;
    return finish(c, rc);
}

int gnb_integrate_cfl(gnb_ctx *c, double t_span, double courant, int max_steps, int mode, double *t_done,
                      int64_t *steps_done)
{
    if (!c) return GNB_EINVAL;
    c->err.clear();
    if (!(t_span >= 0.0) || !std::isfinite(t_span) || !(courant > 0.0) || max_steps < 0)
        return fail(c, GNB_EINVAL, "t_span, courant or max_steps");
    if (!mode_ok(mode)) return fail(c, GNB_EINVAL, "gravity mode");
    if (!c->have_particles) return fail(c, GNB_ESTATE, "no particles");
    if (c->n_gas == 0) return fail(c, GNB_ESTATE, "no gas: the CFL timestep is undefined");
    int rc = GNB_OK;
    if (!c->force_valid || c->last_grav_mode != mode) rc = do_forces(c, mode);
    double t = 0.0;
    int64_t steps = 0;
    while (rc == GNB_OK && t < t_span && steps < max_steps) {
        double m = 0.0;
        rc = cfl_min_h_over_vsig(c, &m);
        if (rc != GNB_OK) break;
        double dt = courant * m;
        if (!(dt > 0.0) || !std::isfinite(dt)) {
            rc = fail(c, GNB_EINVAL, "CFL timestep is not positive");
            break;
        }
        if (dt > t_span - t) dt = t_span - t;
        rc = kdk_one(c, dt, mode);
        t += dt;
        steps++;
    }
    if (t_done) *t_done = t;
    if (steps_done) *steps_done = steps;
    if (rc == GNB_OK) rc = read_groups(c);
    return finish(c, rc);
}

int gnb_integrate_hier(gnb_ctx *c, double t_span, double courant, int max_level, int max_steps, int mode,
                       double *t_done, int64_t info[3])
{
    if (!c) return GNB_EINVAL;
    c->err.clear();
    if (!(t_span > 0.0) || !std::isfinite(t_span) || !(courant > 0.0) || !std::isfinite(courant) || max_level < 1 ||
        max_level > 40 || max_steps < 0)
        return fail(c, GNB_EINVAL, "t_span, courant, max_level or max_steps");
    if (!mode_ok(mode)) return fail(c, GNB_EINVAL, "gravity mode");
    if (!c->have_particles) return fail(c, GNB_ESTATE, "no particles");
    if (c->n_gas == 0) return fail(c, GNB_ESTATE, "no gas: the CFL timestep is undefined");
    if (c->sna_pending) return fail(c, GNB_ESTATE, "an asynchronous surrogate batch is pending");
    c->hier_on = c->hier_valid = false;
    int rc = hier_buffers(c);
    if (rc == GNB_OK && (!c->force_valid || c->last_grav_mode != mode)) rc = do_forces(c, mode);
    const int K = max_level;
    const long long NT = 1ll << (K + 1);
    const double tick = std::ldexp(t_span, -(K + 1));
    long long T = 0;
    int64_t steps = 0, updates = 0, wakes = 0;
    const char *coarse = "a CFL step is shorter than the finest level's (raise max_level)";
    if (rc == GNB_OK) {
        c->hier_on = true;  // from here every sort permutes the step state
        rc = hier_start(c, K, tick, courant, t_span);
    }
    if (rc == GNB_OK && c->hred_h[3]) rc = fail(c, GNB_ECAPACITY, coarse);
    while (rc == GNB_OK && T < NT && steps < max_steps) {
        const long long Tn = (long long)c->hred_h[0];
        const double dd = (double)Tn * tick - (double)T * tick;
        T = Tn;
        phase_begin(c, GNB_T_KDK);
        rc = drift(c, dd);
        if (rc == GNB_OK) rc = hier_predict(c, T, tick);
        phase_end(c);
        c->sorted_valid = c->tree_valid = c->gravity_valid = c->density_valid = c->force_valid = c->sphf_valid = false;
        c->use_pred = true;
        if (rc == GNB_OK) rc = do_forces(c, mode);
        c->use_pred = false;
        phase_begin(c, GNB_T_KDK);
        if (rc == GNB_OK) rc = hier_update(c, T, K, tick, courant, t_span);
        phase_end(c);
        if (rc == GNB_OK && c->hred_h[3]) rc = fail(c, GNB_ECAPACITY, coarse);
        if (rc != GNB_OK) break;
        steps++;
        updates += (int64_t)c->hred_h[1];
        wakes += (int64_t)c->hred_h[2];
    }
    c->hier_valid = rc == GNB_OK;
    if (t_done) *t_done = (double)T * tick;
    if (info) {
        info[0] = steps;
        info[1] = updates;
        info[2] = wakes;
    }
    if (rc == GNB_OK) rc = read_groups(c);
    return finish(c, rc);
}

int gnb_voxelise(gnb_ctx *c, int nreg, const double *centers, double side, int grid, float *out, int on_device)
{
    if (!c) return GNB_EINVAL;
    c->err.clear();
    if (nreg < 1 || !centers || !out || !(side > 0.0) || grid < 1 || grid > 256)
        return fail(c, GNB_EINVAL, "regions, side or grid");
    if (!c->density_valid) return fail(c, GNB_ESTATE, "SPH density not computed for the current positions");
    if (c->sna_pending) return fail(c, GNB_ESTATE, "an asynchronous surrogate batch is pending");
    int rc = voxelise(c, nreg, centers, side, grid, on_device ? out : nullptr);
    if (rc == GNB_OK && !on_device)
        rc = cuda_check(c, cudaMemcpyAsync(out, c->vout, sizeof(float) * 5 * (size_t)nreg * grid * grid * grid,
                                           cudaMemcpyDeviceToHost, c->s), "voxel copy");
    return finish(c, rc);
}

int gnb_remap_regions(gnb_ctx *c, int nreg, const double *centers, double side, int grid, const float *pred,
                      uint64_t seed, int sweeps, int on_device)
{
    if (!c) return GNB_EINVAL;
    c->err.clear();
    if (nreg < 1 || !centers || !pred || !(side > 0.0) || grid < 1 || grid > 256 || sweeps < 0)
        return fail(c, GNB_EINVAL, "regions, side, grid or sweeps");
    if (!c->have_particles) return fail(c, GNB_ESTATE, "no particles");
    if (c->sna_pending) return fail(c, GNB_ESTATE, "an asynchronous surrogate batch is pending");
    const float *pd = pred;
    int rc = GNB_OK;
    if (!on_device) {
        rc = voxelise_buffers_for(c, nreg, grid);
        if (rc == GNB_OK)
            rc = cuda_check(c, cudaMemcpyAsync(c->vout, pred, sizeof(float) * 5 * (size_t)nreg * grid * grid * grid,
                                               cudaMemcpyHostToDevice, c->s), "prediction copy");
        pd = c->vout;
    }
    if (rc == GNB_OK) rc = remap_regions(c, nreg, centers, side, grid, pd, seed, sweeps);
    c->sorted_valid = c->tree_valid = c->gravity_valid = c->density_valid = c->force_valid = c->sphf_valid = false;
    return finish(c, rc);
}

int gnb_sn_surrogate_batch(gnb_ctx *c, gnb_unet *net, int nreg, const double *centers, double side, uint64_t seed,
                           int sweeps, int use_graph)
{
    if (!c) return GNB_EINVAL;
    c->err.clear();
    if (!net || nreg < 1 || !centers || !(side > 0.0) || sweeps < 0) return fail(c, GNB_EINVAL, "arguments");
    if (!c->density_valid) return fail(c, GNB_ESTATE, "SPH density not computed for the current positions");
    if (c->sna_pending) return fail(c, GNB_ESTATE, "an asynchronous surrogate batch is pending");
    int rc = sn_surrogate_batch(c, net, nreg, centers, side, seed, sweeps, use_graph);
    c->sorted_valid = c->tree_valid = c->gravity_valid = c->density_valid = c->force_valid = c->sphf_valid = false;
    rc = finish(c, rc);
    if (rc == GNB_OK && unet_poll_error(net) != GNB_OK)
        return fail(c, GNB_ETIMEOUT, "a bounded wait in the U-Net's tensor-core convolution ran out");
    return rc;
}

int gnb_replace_region(gnb_ctx *c, int64_t n, const int64_t *id, const double *x, const double *y, const double *z,
                       const float *vx, const float *vy, const float *vz, const float *u, int on_device)
{
    if (!c) return GNB_EINVAL;
    c->err.clear();
    if (n < 1) return fail(c, GNB_EINVAL, "particle count out of range");
    if (!id || !x || !y || !z || !vx || !vy || !vz || !u) return fail(c, GNB_EINVAL, "null array");
    if (!c->have_particles) return fail(c, GNB_ESTATE, "no particles");
    if (c->sna_pending) return fail(c, GNB_ESTATE, "an asynchronous surrogate batch is pending");
    if (n > c->n) return fail(c, GNB_EMISMATCH, "more particles than the context holds");
    int rc = replace_particles(c, n, id, x, y, z, vx, vy, vz, u, on_device);
    if (rc == GNB_OK)
        c->sorted_valid = c->tree_valid = c->gravity_valid = c->density_valid = c->force_valid = c->sphf_valid = false;
    return finish(c, rc);
}

static int64_t field_count(gnb_ctx *c, int f, size_t *esz)
{
    switch (f) {
    case GNB_F_X: case GNB_F_Y: case GNB_F_Z: case GNB_F_H2: *esz = 8; return c->n;
    case GNB_F_KEY: case GNB_F_ORDER: case GNB_F_ID: *esz = 8; return c->n;
    case GNB_F_NBR: *esz = 8; return c->n_gas * 64;
    case GNB_F_NODES: *esz = 8; return 4 * (int64_t)c->t.nnodes;
    case GNB_F_NODE_LINKS: *esz = 8; return 3 * (int64_t)c->t.nnodes;
    case GNB_F_GROUPS: *esz = 8; return c->t.ngroups;
    default: *esz = 4; return c->n;
    }
}

// Whether `field` holds current values (GNB_OK) or why not.
static int field_ready(gnb_ctx *c, int field)
{
    if (field < 0 || field >= GNB_F_COUNT_) return fail(c, GNB_EINVAL, "field");
    bool need_sort = field == GNB_F_KEY || field == GNB_F_ORDER;
    bool need_tree = field == GNB_F_NODES || field == GNB_F_NODE_LINKS || field == GNB_F_GROUPS;
    bool need_grav = field == GNB_F_AX || field == GNB_F_AY || field == GNB_F_AZ || field == GNB_F_POT ||
                     field == GNB_F_POT_EXT ||
                     field == GNB_F_AGRAV_X || field == GNB_F_AGRAV_Y || field == GNB_F_AGRAV_Z;
    bool need_den = field == GNB_F_RHO || field == GNB_F_PRES || field == GNB_F_CS || field == GNB_F_NBR;
    if (need_sort && !c->sorted_valid) return fail(c, GNB_ESTATE, "particles not sorted for the current positions");
    if (need_tree && !c->tree_valid) return fail(c, GNB_ESTATE, "tree not built");
    bool total_acc = field == GNB_F_AX || field == GNB_F_AY || field == GNB_F_AZ;
    // the total acceleration, du/dt and the supports are also current when
    // they came with the state (gnb_set_state)
    if (need_grav && !c->gravity_valid && !(total_acc && (c->sphf_valid || c->force_valid)))
        return fail(c, GNB_ESTATE, "forces not computed");
    if (need_den && !c->density_valid) return fail(c, GNB_ESTATE, "SPH density not computed");
    if (field == GNB_F_H2 && !c->density_valid && !(c->have_h && c->force_valid))
        return fail(c, GNB_ESTATE, "SPH density not computed");
    if (field == GNB_F_NBR && !c->nbr_valid) return fail(c, GNB_ESTATE, "neighbour lists not computed");
    if (field == GNB_F_DUDT && !c->sphf_valid && !c->force_valid) return fail(c, GNB_ESTATE, "SPH force not computed");
    if (field == GNB_F_LEVEL && !c->hier_valid) return fail(c, GNB_ESTATE, "no hierarchical integration");
    return GNB_OK;
}

int gnb_get(gnb_ctx *c, int field, void *dst, int64_t cap, int on_device)
{
    if (!c) return GNB_EINVAL;
    c->err.clear();
    if (!dst || field < 0 || field >= GNB_F_COUNT_) return fail(c, GNB_EINVAL, "field or destination");
    if (!c->have_particles) return fail(c, GNB_ESTATE, "no particles");
    GNB_TRY(field_ready(c, field));
    size_t esz;
    int64_t cnt = field_count(c, field, &esz);
    if (cap < cnt) return fail(c, GNB_EINVAL, "destination too small");
    if (cnt == 0) return GNB_OK;
    int rc;
    if (on_device) {
        rc = scatter_out(c, field, dst);
    } else {
        void *tmp = c->tmp_out;
        bool own = false;
        if ((size_t)cnt * esz > (size_t)c->cap * 8 + 64) {  // the staging buffer holds 8 cap + 64 bytes
            if (cudaMalloc(&tmp, (size_t)cnt * esz) != cudaSuccess) return fail(c, GNB_ENOMEM, "export buffer");
            own = true;
        }
        rc = scatter_out(c, field, tmp);
        if (rc == GNB_OK)
            rc = cuda_check(c, cudaMemcpyAsync(dst, tmp, (size_t)cnt * esz, cudaMemcpyDeviceToHost, c->s), "export copy");
        if (rc == GNB_OK) rc = cuda_check(c, cudaStreamSynchronize(c->s), "export sync");
        if (own) cudaFree(tmp);
    }
    return finish(c, rc);
}

int gnb_get_fields(gnb_ctx *c, int nf, const int *fields, void *const *dst, const int64_t *cap, int on_device)
{
    if (!c) return GNB_EINVAL;
    c->err.clear();
    if (nf < 0 || (nf > 0 && (!fields || !dst || !cap))) return fail(c, GNB_EINVAL, "field list");
    if (!c->have_particles) return fail(c, GNB_ESTATE, "no particles");
    // every field is checked before any is copied
    std::vector<int64_t> cnt((size_t)nf);
    std::vector<size_t> esz((size_t)nf);
    size_t big = 0;
    for (int k = 0; k < nf; k++) {
        if (!dst[k] || fields[k] < 0 || fields[k] >= GNB_F_COUNT_) return fail(c, GNB_EINVAL, "field or destination");
        GNB_TRY(field_ready(c, fields[k]));
        cnt[k] = field_count(c, fields[k], &esz[k]);
        if (cap[k] < cnt[k]) return fail(c, GNB_EINVAL, "destination too small");
        big = std::max(big, (size_t)cnt[k] * esz[k]);
    }
    // host destinations: every field through the one staging buffer, its
    // copy queued behind its gather on the stream (the next gather waits for
    // it there), one synchronisation for all
    void *tmp = c->tmp_out;
    bool own = false;
    if (!on_device && big > (size_t)c->cap * 8 + 64) {
        if (cudaMalloc(&tmp, big) != cudaSuccess) return fail(c, GNB_ENOMEM, "export buffer");
        own = true;
    }
    int rc = GNB_OK;
    for (int k = 0; k < nf && rc == GNB_OK; k++) {
        if (cnt[k] == 0) continue;
        if (on_device) {
            rc = scatter_out(c, fields[k], dst[k]);
        } else {
            rc = scatter_out(c, fields[k], tmp);
            if (rc == GNB_OK)
                rc = cuda_check(c, cudaMemcpyAsync(dst[k], tmp, (size_t)cnt[k] * esz[k], cudaMemcpyDeviceToHost, c->s),
                                "export copy");
        }
    }
    if (rc == GNB_OK && !on_device) rc = cuda_check(c, cudaStreamSynchronize(c->s), "export sync");
    if (own) cudaFree(tmp);
    return finish(c, rc);
}

int gnb_save(gnb_ctx *c, const char *path)
{
    if (!c || !path) return GNB_EINVAL;
    c->err.clear();
    if (!c->have_particles) return fail(c, GNB_ESTATE, "no particles");
    if (c->sna_pending) return fail(c, GNB_ESTATE, "an asynchronous surrogate batch is pending");
    return finish(c, save_state(c, path));
}

int gnb_load(gnb_ctx *c, const char *path)
{
    if (!c || !path) return GNB_EINVAL;
    c->err.clear();
    return finish(c, load_state(c, path));
}

int gnb_diagnostics(gnb_ctx *c, double out[10])
{
    if (!c || !out) return GNB_EINVAL;
    c->err.clear();
    if (!c->gravity_valid) return fail(c, GNB_ESTATE, "forces not computed");
    return finish(c, diagnostics(c, out));
}

int gnb_stats(gnb_ctx *c, int64_t out[GNB_S_COUNT_])
{
    if (!c || !out) return GNB_EINVAL;
    unsigned long long h[2] = {0, 0};
    if (c->counters_d) {
        cudaStreamSynchronize(c->s);
        cudaMemcpy(h, c->counters_d, sizeof(h), cudaMemcpyDeviceToHost);
    }
    c->stats[GNB_S_NPP] = (int64_t)h[0];
    c->stats[GNB_S_NPC] = (int64_t)h[1];
    int rt = 0;
    if (c->rtot_d && c->n_gas > 0) cudaMemcpy(&rt, c->rtot_d, sizeof(int), cudaMemcpyDeviceToHost);
    c->stats[GNB_S_NSYM] = (int64_t)c->n_gas * 63 + rt;
    for (int k = 0; k < GNB_S_COUNT_; k++) out[k] = c->stats[k];
    return GNB_OK;
}

int gnb_set_timing(gnb_ctx *c, int enable)
{
    if (!c) return GNB_EINVAL;
    phase_resolve(c);
    c->timing = enable != 0;
    return GNB_OK;
}

int gnb_sn_async_submit(gnb_ctx *c, gnb_unet *net, int nreg, const double *centers, double side, uint64_t seed,
                        int sweeps)
{
    if (!c) return GNB_EINVAL;
    c->err.clear();
    if (!net || nreg < 1 || !centers || !(side > 0.0) || sweeps < 0) return fail(c, GNB_EINVAL, "arguments");
    if (!c->density_valid) return fail(c, GNB_ESTATE, "SPH density not computed for the current positions");
    int rc = sn_async_submit(c, net, nreg, centers, side, seed, sweeps);
    return finish(c, rc);
}

int gnb_sn_async_apply(gnb_ctx *c)
{
    if (!c) return GNB_EINVAL;
    c->err.clear();
    int rc = sn_async_apply(c);
    if (rc == GNB_OK) c->sorted_valid = c->tree_valid = c->gravity_valid = c->density_valid = c->force_valid = c->sphf_valid = false;
    rc = finish(c, rc);
    if (rc == GNB_OK && unet_poll_error((gnb_unet *)c->sna_net) != GNB_OK)
        return fail(c, GNB_ETIMEOUT, "a bounded wait in the U-Net's tensor-core convolution ran out");
    return rc;
}

int gnb_sn_async_pending(const gnb_ctx *c) { return c && c->sna_pending ? 1 : 0; }

int gnb_set_sn_chunks(gnb_ctx *c, int chunks)
{
    if (!c || chunks < 1 || chunks > gnb_ctx::SN_MAXCH) return GNB_EINVAL;
    c->sn_chunks = chunks;
    return GNB_OK;
}

int gnb_phase_times(gnb_ctx *c, double out_ms[GNB_T_COUNT_], int64_t calls[GNB_T_COUNT_], int64_t *launches,
                    int reset)
{
    if (!c) return GNB_EINVAL;
    cudaStreamSynchronize(c->s);
    phase_resolve(c);
    for (int k = 0; k < GNB_T_COUNT_; k++) {
        if (out_ms) out_ms[k] = c->phase_ms[k];
        if (calls) calls[k] = c->phase_calls[k];
    }
    long long now = g_launches.load();
    if (launches) *launches = now - c->launch_base;
    if (reset) {
        for (int k = 0; k < GNB_T_COUNT_; k++) { c->phase_ms[k] = 0; c->phase_calls[k] = 0; }
        c->launch_base = now;
    }
    return GNB_OK;
}

const char *gnb_last_error(const gnb_ctx *c)
{
    if (!c) return "null context";
    return c->err.c_str();
}

}  // extern "C"
