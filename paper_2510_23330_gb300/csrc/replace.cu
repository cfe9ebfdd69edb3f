// replace.cu -- replacement of particles by ID (gnb_replace_region in galnb.h).
//
// Sec. 3.2, step 4: the nodes integrating the galaxy overwrite the particles
// that the surrogate (or any other integrator of a supernova region) hands
// back, matched on their particle IDs.  The library keeps its particles in
// Morton order and re-sorts them every step, so an ID is found in two steps:
//   1. the held IDs, sorted with their caller indices (built once after
//      gnb_set_particles; IDs and caller indices do not change until the
//      next gnb_set_particles), give the caller index of an ID by binary
//      search;
//   2. the inverse of the slot -> caller-index permutation of the current
//      order gives the slot.
// A first kernel checks every incoming particle (ID held exactly once, not
// repeated in the input, finite position) without touching the particles;
// only when all pass does a second kernel write them, so a rejected call
// leaves the state as it was.
#include "common.cuh"

namespace gnb {

enum : int { RP_UNKNOWN = 1, RP_AMBIGUOUS = 2, RP_DUPLICATE = 4, RP_NONFINITE = 8 };

__global__ void k_rid_init(const int64_t *__restrict__ id, const int *__restrict__ orig, int n,
                           uint64_t *__restrict__ key, int *__restrict__ val)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    key[i] = (uint64_t)id[i];  // the order of the bit patterns serves the search; it need not be numeric
    val[i] = orig[i];
}

__global__ void k_rid_inverse(const int *__restrict__ orig, int n, int *__restrict__ inv, int *__restrict__ mark)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    inv[orig[i]] = i;
    mark[i] = 0;
}

struct RepIn {
    const int64_t *id;
    const double *x, *y, *z;
    const float *vx, *vy, *vz, *u;
};

__global__ void k_rep_check(RepIn in, int m, const uint64_t *__restrict__ rkey, const int *__restrict__ rorig,
                            int n, const int *__restrict__ inv, int *__restrict__ mark, int *__restrict__ slot,
                            int *__restrict__ flag)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    uint64_t q = (uint64_t)in.id[j];
    int lo = 0, hi = n;  // first entry >= q
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (rkey[mid] < q) lo = mid + 1;
        else hi = mid;
    }
    int f = 0;
    if (lo >= n || rkey[lo] != q) {
        f |= RP_UNKNOWN;
    } else {
        if (lo + 1 < n && rkey[lo + 1] == q) f |= RP_AMBIGUOUS;
        int o = rorig[lo];
        if (atomicAdd(&mark[o], 1) != 0) f |= RP_DUPLICATE;
        slot[j] = inv[o];
    }
    if (!isfinite(in.x[j]) || !isfinite(in.y[j]) || !isfinite(in.z[j])) f |= RP_NONFINITE;
    if (f) atomicOr(flag, f);
}

__global__ void k_rep_write(RepIn in, int m, const int *__restrict__ slot, PArr p)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    int s = slot[j];
    p.x[s] = in.x[j]; p.y[s] = in.y[j]; p.z[s] = in.z[j];
    float vx = in.vx[j], vy = in.vy[j], vz = in.vz[j];
    p.vx[s] = vx; p.vy[s] = vy; p.vz[s] = vz;
    p.vpx[s] = vx; p.vpy[s] = vy; p.vpz[s] = vz;
    if (p.type[s] == GNB_GAS) {
        float u = in.u[j];
        p.u[s] = u;
        p.up[s] = u;
    }
}

void replace_free(gnb_ctx *c)
{
    void *all[] = {c->rid_key, c->rid_key2, c->rid_orig, c->rid_orig2, c->rid_inv, c->rid_mark, c->rep_buf,
                   c->rep_slot};
    for (void *q : all) dfree(c, q);
    c->rid_key = c->rid_key2 = nullptr;
    c->rid_orig = c->rid_orig2 = c->rid_inv = c->rid_mark = c->rep_slot = nullptr;
    c->rep_buf = nullptr;
    c->rid_cap = c->rep_cap = c->rep_scap = 0;
    c->rid_valid = false;
}

int replace_particles(gnb_ctx *c, int64_t m64, const int64_t *id, const double *x, const double *y, const double *z,
                      const float *vx, const float *vy, const float *vz, const float *u, int on_device)
{
    int n = (int)c->n;
    int m = (int)m64;
    if (c->rid_cap < c->n) {
        dfree(c, c->rid_key); dfree(c, c->rid_key2); dfree(c, c->rid_orig); dfree(c, c->rid_orig2);
        dfree(c, c->rid_inv); dfree(c, c->rid_mark);
        c->rid_key = c->rid_key2 = nullptr;
        c->rid_orig = c->rid_orig2 = c->rid_inv = c->rid_mark = nullptr;
        c->rid_cap = 0;
        c->rid_valid = false;
        size_t N = (size_t)c->n;
        GNB_TRY(dalloc(c, &c->rid_key, N)); GNB_TRY(dalloc(c, &c->rid_key2, N));
        GNB_TRY(dalloc(c, &c->rid_orig, N)); GNB_TRY(dalloc(c, &c->rid_orig2, N));
        GNB_TRY(dalloc(c, &c->rid_inv, N)); GNB_TRY(dalloc(c, &c->rid_mark, N));
        c->rid_cap = c->n;
    }
    int nb = (n + 255) / 256;
    PArr &p = c->P[c->cur];
    if (!c->rid_valid) {
        gnb::counted(k_rid_init)<<<nb, 256, 0, c->s>>>(p.id, p.orig, n, c->rid_key, c->rid_orig);
        GNB_LAUNCH_CHECK(c, "replace: ID table");
        GNB_TRY(radix_sort_pairs(c, c->rid_key, c->rid_orig, c->rid_key2, c->rid_orig2, n, 0));
        c->rid_valid = true;
    }
    gnb::counted(k_rid_inverse)<<<nb, 256, 0, c->s>>>(p.orig, n, c->rid_inv, c->rid_mark);
    if (c->rep_scap < m64) {
        dfree(c, c->rep_slot);
        c->rep_slot = nullptr;
        c->rep_scap = 0;
        GNB_TRY(dalloc(c, &c->rep_slot, (size_t)m));
        c->rep_scap = m64;
    }
    RepIn in{id, x, y, z, vx, vy, vz, u};
    if (!on_device) {
        if (c->rep_cap < m64) {
            dfree(c, c->rep_buf);
            c->rep_buf = nullptr;
            c->rep_cap = 0;
            GNB_TRY(dalloc(c, &c->rep_buf, (size_t)m * 48 + 256));
            c->rep_cap = m64;
        }
        unsigned char *b = c->rep_buf;
        size_t M = (size_t)m;
        int64_t *did = (int64_t *)b;
        double *dx = (double *)(b + 8 * M), *dy = dx + M, *dz = dy + M;
        float *dvx = (float *)(dz + M), *dvy = dvx + M, *dvz = dvy + M, *du = dvz + M;
        struct { void *d; const void *s; size_t bytes; } cp[] = {
            {did, id, 8 * M}, {dx, x, 8 * M}, {dy, y, 8 * M}, {dz, z, 8 * M},
            {dvx, vx, 4 * M}, {dvy, vy, 4 * M}, {dvz, vz, 4 * M}, {du, u, 4 * M}};
        for (auto &q : cp)
            GNB_TRY(cuda_check(c, cudaMemcpyAsync(q.d, q.s, q.bytes, cudaMemcpyHostToDevice, c->s), "replace: copy"));
        in = RepIn{did, dx, dy, dz, dvx, dvy, dvz, du};
    }
    cudaMemsetAsync(c->work_d, 0, sizeof(int), c->s);
    int mb = (m + 255) / 256;
    gnb::counted(k_rep_check)<<<mb, 256, 0, c->s>>>(in, m, c->rid_key, c->rid_orig, n, c->rid_inv, c->rid_mark,
                                                    c->rep_slot, c->work_d);
    GNB_LAUNCH_CHECK(c, "replace: check");
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(c->pinned_i, c->work_d, sizeof(int), cudaMemcpyDeviceToHost, c->s),
                       "replace: flag"));
    GNB_TRY(cuda_check(c, cudaStreamSynchronize(c->s), "replace: sync"));
    int f = c->pinned_i[0];
    if (f & RP_UNKNOWN) return fail(c, GNB_EMISMATCH, "an ID is not held by the context");
    if (f & RP_AMBIGUOUS) return fail(c, GNB_EMISMATCH, "an ID is held by more than one particle");
    if (f & RP_DUPLICATE) return fail(c, GNB_EMISMATCH, "an ID appears more than once in the input");
    if (f & RP_NONFINITE) return fail(c, GNB_EINVAL, "non-finite position");
    gnb::counted(k_rep_write)<<<mb, 256, 0, c->s>>>(in, m, c->rep_slot, p);
    GNB_LAUNCH_CHECK(c, "replace: write");
    return GNB_OK;
}

}  // namespace gnb
