// sph.cu -- SPH kernel size, density/pressure and hydro force
// (Sec. 5.2.5, Table 3 "kernel size", "density and pressure", "hydro force"
// and Table 4 of Hirashima et al., SC'25).
//
// Kernel size: the support h_i of gas particle i is the distance to its
// n_ngb-th nearest gas neighbour (self included), neighbours ordered by
// (d^2, gas rank) with d^2 = (dx*dx + dy*dy) + dz*dz in FP64.  The paper
// iterates a search until it converges; here one CTA per hydro-tree group
// gathers every gas particle within a search radius R of the group into
// shared memory, and each warp selects the neighbours of one particle:
//   1. FP32 distances d from FP32 offsets to the group's reference cell,
//      with |d - D| <= E(D) = 2^-23 (4 sqrt(3) A' sqrt(D) + 5 D), A' = the
//      largest offset in the group plus two grid units: each offset carries
//      one rounding (<= 2^-24 A') plus the residual's (<= 2^-24 unit), the
//      difference and the three fused multiply-adds one rounding each, and
//      the factor 2 over the first-order bound covers the second-order terms,
//   2. a 64-bin histogram and an in-bucket rank give the exact 64th smallest
//      FP32 value t,
//   3. entries with d < t - 2E are certainly neighbours, entries with
//      d > t + 2E certainly not; only the few in between get the exact FP64
//      d^2 and are ranked by (d^2, gas rank).
// A group whose radius holds fewer than n_ngb particles for some member
// retries with a larger radius (bisected once both bounds are known: the
// paper's "usually twice"); a group whose candidates do not fit is split into
// single-particle items, and a single particle whose candidates do not fit
// retries with a smaller radius.  Each pass hands the next only its
// unfinished items.  Density and the ideal-gas EOS are fused in.
//
// Force: symmetric SPH over S_i = N_i u {j : i in N_j}.  The reverse part is
// built from the non-mutual pairs only, so N_i and R_i are disjoint.
#include "common.cuh"

namespace gnb {

#define KN_THREADS 128
#define KN_WARPS (KN_THREADS / 32)
// Candidate buffer and node stack size the shared memory of a CTA (24.7 KB),
// and with it the CTAs per SM (9, as the 56 registers allow).
#define KN_CAP 768
#define KN_STACK 768
#define KN_BKT 256
#define KN_U 64
#define KN_SUB 4  // particles per work item when a group splits (2^24 disk: 6.52 ms for the pass, 8: 6.77, singles: 7.05)
#define NGB 64

__device__ __forceinline__ float kern_w(float r, float hinv)
{
    float q = r * hinv;
    float s = 2.546479089470325f * hinv * hinv * hinv;  // 8/pi h^-3
    if (q <= 0.5f) return s * (1.f - 6.f * q * q + 6.f * q * q * q);
    if (q <= 1.f) { float t = 1.f - q; return s * 2.f * t * t * t; }
    return 0.f;
}

__device__ __forceinline__ float kern_dw(float r, float hinv)
{
    float q = r * hinv;
    float s = 2.546479089470325f * hinv * hinv * hinv * hinv;
    if (q <= 0.5f) return s * (-12.f * q + 18.f * q * q);
    if (q <= 1.f) { float t = 1.f - q; return -6.f * s * t * t; }
    return 0.f;
}

// ---------------------------------------------------------------- gas extraction
struct GasGather {
    const uint64_t *skey;
    PArr p;
    const int *gslot;
    uint64_t *gkey;
    int *gcx, *gcy, *gcz, *ggrank;
    float *grx, *gry, *grz, *gm, *gvx, *gvy, *gvz, *gu, *gRprev;
    double *gx, *gy, *gz;
    int ng;
    int pred;
    int have_h;
};

__global__ void k_gas_gather(GasGather g)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.ng) return;
    int s = g.gslot[k];
    g.gkey[k] = g.skey[s];
    g.gcx[k] = g.p.cx[s]; g.gcy[k] = g.p.cy[s]; g.gcz[k] = g.p.cz[s];
    g.grx[k] = g.p.rx[s]; g.gry[k] = g.p.ry[s]; g.grz[k] = g.p.rz[s];
    g.gx[k] = g.p.x[s]; g.gy[k] = g.p.y[s]; g.gz[k] = g.p.z[s];
    g.gm[k] = g.p.m[s];
    g.ggrank[k] = g.p.grank[s];
    if (g.pred) {
        g.gvx[k] = g.p.vpx[s]; g.gvy[k] = g.p.vpy[s]; g.gvz[k] = g.p.vpz[s]; g.gu[k] = g.p.up[s];
    } else {
        g.gvx[k] = g.p.vx[s]; g.gvy[k] = g.p.vy[s]; g.gvz[k] = g.p.vz[s]; g.gu[k] = g.p.u[s];
    }
    g.gRprev[k] = g.have_h ? sqrtf((float)g.p.h2[s]) : 0.f;  // a starting radius only
}

// ---------------------------------------------------------------- search radius
// Initial radius per hydro group: margin x the largest previous support in
// the group, or, without history, a density estimate from the smallest
// ancestor cell holding at least n_ngb particles.  A group split into
// single-particle items gives each particle margin x its own previous
// support (at most the group's radius).  The margin trades retried items (a
// support that grew past it) against candidates per item (the search volume
// grows as its cube); the host adapts it to the retries it sees (see
// sph_density).
__global__ void k_knn_init(Tree t, const float *__restrict__ hprev, int have_h, float margin, const double *__restrict__ box,
                           float *__restrict__ kR, float2 *__restrict__ kRb, int *__restrict__ kflag,
                           int2 *__restrict__ kitem, int *__restrict__ nitems)
{
    int ng = *t.ngroups_d;
    float unit = (float)box[4];
    if (blockIdx.x == 0 && threadIdx.x == 0) *nitems = ng;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        int node = t.groups[g];
        int4 a = t.na[node];
        kitem[g] = make_int2(a.x, a.y);
        float R = 0.f;
        if (have_h) {
            for (int i = a.x; i < a.x + a.y; i++) R = fmaxf(R, hprev[i]);
            R *= margin;
        }
        if (!(R > 0.f)) {
            int q = node;
            while (t.na[q].y < NGB && t.nb[q].w >= 0) q = t.nb[q].w;
            int4 aq = t.na[q];
            int lev = aq.w & 255;
            float side = (float)(1 << (GNB_MAXLEV - lev)) * unit;
            R = 0.9f * side * cbrtf((float)NGB / (float)max(aq.y, 1));
        }
        kR[g] = R;
        kRb[g] = make_float2(0.f, 0.f);
        kflag[g] = 1;
    }
}

// Work items: a hydro group, or a single particle split off a group whose
// candidates did not fit at the radius its members need.
struct KnnParams {
    int4 *na, *nb;
    int2 *item;
    int *nitems;       // live count (splits append here)
    const int *nsnap;  // entries of this pass's worklist
    const int *wl_in;  // this pass's items (null: items 0 .. *nsnap - 1)
    int *wl_out;       // items left for the next pass: retried radii and new single-particle items
    int *nwl_out;
    int item_cap;
    const int *gcx, *gcy, *gcz, *ggrank;
    const float *grx, *gry, *grz, *gm, *gu;
    const double *gx, *gy, *gz;
    const double *box;
    const float *rprev;  // previous support per gas particle (0: none)
    float margin;        // search radius over the previous support
    int *nunder;         // work items whose radius held too few candidates
    float *kR;
    float2 *kRb;
    int *kflag;
    int *next;
    int *remaining;
    int *status;
    int *nbr;
    float *nd2;
    double *h2;
    float *h2lo, *h2hi;
    float *h, *E, *rho, *P, *cs;
    int *g64;
    float gamma;
    int pressure;  // 1: also smooth P = (gamma - 1) sum_j m_j u_j W_ij (pressure-energy SPH)
};

struct KnnSmem {
    float4 cand[KN_CAP];
    int stack[KN_STACK];
    int hist[KN_WARPS][64];
    float bkt[KN_WARPS][KN_BKT];
    int bn[KN_WARPS];
    int un[KN_WARPS];
    int ui[KN_WARPS][KN_U];
    long long uD[KN_WARPS][KN_U];  // exact FP64 d^2 as bit patterns (non-negative: they order like the values)
    int ug[KN_WARPS][KN_U];        // gas ranks of the uncertain entries
    int nc, sp, g, wb, under, over, split, nleaf, bmin[3], bmax[3];
    long long rg2i;
    unsigned amax;
};
// During the gather the bucket buffers hold the list of leaves within the
// radius (first, count) and its prefix sums over the counts.
#define KN_LEAF 256
static_assert(sizeof(float) * KN_WARPS * KN_BKT >= (sizeof(int2) + sizeof(int)) * KN_LEAF + sizeof(int),
              "leaf list must fit the bucket buffers");

// A particle of a group could not be ranked within the buffers: the FP32
// error band (2^-17 A^2, A the group's largest offset) is wide when a dense
// clump sits inside a spread-out group.  The group is then split into
// single-particle work items, whose band scales with their own search
// radius; only a single particle that still fails is reported.
__device__ __forceinline__ void knn_fail(KnnSmem &S, int count, int *status)
{
    if (count > 1) S.split = 1;
    else atomicOr(status, ST_KNN_OVERFLOW);
}

__device__ __forceinline__ float d2f(float4 c, float xi, float yi, float zi)
{
    float dx = c.x - xi, dy = c.y - yi, dz = c.z - zi;
    return __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, dz * dz));
}

__device__ __forceinline__ double exact_d2(const double *x, const double *y, const double *z, int i, int j)
{
    double dx = __dsub_rn(x[i], x[j]), dy = __dsub_rn(y[i], y[j]), dz = __dsub_rn(z[i], z[j]);
    double a = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    return __dadd_rn(a, __dmul_rn(dz, dz));
}

// Exact k-th smallest FP32 d^2 (1-based k) among the candidates of this
// warp's particle that fall in histogram bucket bstar of [0, R2sel] (the
// same bin rule as the histogram): a radix select on the bit patterns, which
// order non-negative floats like their values, 8 bits per pass.  Used when
// the bucket holds more candidates than the bucket buffer -- a particle whose
// nearest neighbours all lie in a thin shell, e.g. a compact clump seen from
// outside, where shrinking the radius does not thin the bucket.
__device__ __noinline__ float knn_radix_kth(KnnSmem &S, int w, int lane, int nc, float xi, float yi, float zi, float R2sel,
                               float inv64, int bstar, int k, bool *ok)
{
    int *hb = reinterpret_cast<int *>(S.bkt[w]);  // 256 bins (the bucket buffer is free here)
    unsigned prefix = 0u, pmask = 0u;
    for (int shift = 24; shift >= 0; shift -= 8) {
        __syncwarp();
        for (int b = lane; b < 256; b += 32) hb[b] = 0;
        __syncwarp();
        for (int c = lane; c < nc; c += 32) {
            const float d = d2f(S.cand[c], xi, yi, zi);
            if (d <= R2sel && min(63, (int)(d * inv64)) == bstar) {
                const unsigned u = __float_as_uint(d);
                if ((u & pmask) == prefix) atomicAdd(&hb[(u >> shift) & 255u], 1);
            }
        }
        __syncwarp();
        int loc[8], sum = 0;
#pragma unroll
        for (int q = 0; q < 8; q++) { loc[q] = hb[8 * lane + q]; sum += loc[q]; }
        int inc = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        const int exc = inc - sum;
        int myb = -1, mybefore = 0, run = exc;
#pragma unroll
        for (int q = 0; q < 8; q++) {
            if (myb < 0 && run < k && k <= run + loc[q]) { myb = 8 * lane + q; mybefore = run; }
            run += loc[q];
        }
        const unsigned bal = __ballot_sync(0xffffffffu, myb >= 0);
        if (bal == 0u) { *ok = false; return 0.f; }
        const int src = __ffs(bal) - 1;
        const int b = __shfl_sync(0xffffffffu, myb, src);
        k -= __shfl_sync(0xffffffffu, mybefore, src);
        prefix |= (unsigned)b << shift;
        pmask |= 255u << shift;
    }
    *ok = true;
    return __uint_as_float(prefix);
}

__global__ void __launch_bounds__(KN_THREADS, 9) k_knn(KnnParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    KnnSmem &S = *reinterpret_cast<KnnSmem *>(smem_raw);
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const float unit = (float)p.box[4];
    const int ngroups = min(*p.nsnap, p.item_cap);
    const unsigned ltmask = (1u << lane) - 1u;
    for (;;) {
        __syncthreads();  // every thread has read the previous S.g
        if (tid == 0) S.g = atomicAdd(p.next, 1);
        __syncthreads();
        if (S.g >= ngroups) break;
        const int gi = p.wl_in ? p.wl_in[S.g] : S.g;
        if (p.kflag[gi] == 0) continue;  // uniform
        const int2 gitem = p.item[gi];
        const int4 ga = make_int4(gitem.x, gitem.y, 0, 0);
        const float R = p.kR[gi];
        if (tid < 3) { S.bmin[tid] = 0x7fffffff; S.bmax[tid] = -1; }
        if (tid == 0) {
            S.nc = 0; S.sp = 1; S.stack[0] = 0; S.under = 0; S.over = 0; S.split = 0; S.amax = 0u; S.nleaf = 0;
            // the node test's threshold: (R in grid units)^2 (1 + 1e-5) + 4, in
            // FP64 by one thread (GB300's FP64 pipe is narrow).  gap2 is an
            // integer, so gap2 <= that exactly when gap2 <= its floor
            const double Rg = (double)R / (double)unit;
            const double Rg2m = Rg * Rg * (1.0 + 1e-5) + 4.0;
            S.rg2i = Rg2m >= 4.0e18 ? 0x7fffffffffffffffll : (long long)Rg2m;
        }
        __syncthreads();
        for (int i = ga.x + tid; i < ga.x + ga.y; i += KN_THREADS) {
            atomicMin(&S.bmin[0], p.gcx[i]); atomicMax(&S.bmax[0], p.gcx[i]);
            atomicMin(&S.bmin[1], p.gcy[i]); atomicMax(&S.bmax[1], p.gcy[i]);
            atomicMin(&S.bmin[2], p.gcz[i]); atomicMax(&S.bmax[2], p.gcz[i]);
        }
        __syncthreads();
        const int b0[3] = {S.bmin[0], S.bmin[1], S.bmin[2]}, b1[3] = {S.bmax[0], S.bmax[1], S.bmax[2]};
        const int gref[3] = {(b0[0] + b1[0]) >> 1, (b0[1] + b1[1]) >> 1, (b0[2] + b1[2]) >> 1};
        // group box in offset coordinates: [lo_k, hi_k)
        float blo[3], bhi[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            blo[a] = (float)(b0[a] - gref[a]) * unit;
            bhi[a] = (float)(b1[a] + 1 - gref[a]) * unit;
        }
        const long long Rg2i = S.rg2i;
        const float R2stage = R * R * (1.f + 1e-4f) + 4.f * unit * unit;
        int2 *leafl = reinterpret_cast<int2 *>(&S.bkt[0][0]);
        int *lpre = reinterpret_cast<int *>(leafl + KN_LEAF);
        // gather candidates within R of the group box: the walk lists the
        // leaves it reaches, then all threads test their particles together
        for (;;) {
            __syncthreads();
            int sp = S.sp;
            if (sp == 0) break;
            int k = min(KN_THREADS, sp);
            int room = (KN_STACK - sp) / 7;
            k = min(k, max(room, 1));
            int node = tid < k ? S.stack[sp - k + tid] : -1;
            __syncthreads();
            if (tid == 0) S.sp = sp - k;
            __syncthreads();
            if (node >= 0) {
                int4 a = p.na[node];
                int4 C = p.nb[node];
                int lev = a.w & 255, nch = a.w >> 8;
                long long s = 1ll << (GNB_MAXLEV - lev);
                int cc[3] = {C.x, C.y, C.z};
                long long gap2 = 0;  // < 3 * 2^44: exact in 64-bit integers
#pragma unroll
                for (int q = 0; q < 3; q++) {
                    long long gp = 0;
                    if ((long long)cc[q] > (long long)b1[q] + 1) gp = cc[q] - ((long long)b1[q] + 1);
                    else if ((long long)b0[q] > cc[q] + s) gp = b0[q] - (cc[q] + s);
                    gap2 += gp * gp;
                }
                if (gap2 <= Rg2i) {
                    if (nch > 0) {
                        int b = atomicAdd(&S.sp, nch);
                        if (b + nch <= KN_STACK) {
                            for (int q = 0; q < nch; q++) S.stack[b + q] = a.z + q;
                        } else {
                            atomicSub(&S.sp, nch);
                            S.over = 1;
                        }
                    } else {
                        const int q = atomicAdd(&S.nleaf, 1);
                        if (q < KN_LEAF) leafl[q] = make_int2(a.x, a.y);
                        else  // the list is full: this thread tests the leaf's particles
                        for (int j = a.x; j < a.x + a.y; j++) {
                            float ox = grid_off(p.gcx[j], gref[0], p.grx[j], unit);
                            float oy = grid_off(p.gcy[j], gref[1], p.gry[j], unit);
                            float oz = grid_off(p.gcz[j], gref[2], p.grz[j], unit);
                            float gx = fmaxf(0.f, fmaxf(blo[0] - ox, ox - bhi[0]));
                            float gy = fmaxf(0.f, fmaxf(blo[1] - oy, oy - bhi[1]));
                            float gz = fmaxf(0.f, fmaxf(blo[2] - oz, oz - bhi[2]));
                            if (gx * gx + gy * gy + gz * gz <= R2stage) {
                                int slot = atomicAdd(&S.nc, 1);
                                if (slot < KN_CAP) {
                                    S.cand[slot] = make_float4(ox, oy, oz, __int_as_float(j));
                                    float a2 = ox * ox + oy * oy + oz * oz;
                                    atomicMax(&S.amax, __float_as_uint(a2));
                                } else {
                                    S.over = 1;
                                }
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();
        {   // the listed leaves' particles, flattened over all threads
            const int nl = min(S.nleaf, KN_LEAF);
            if (w == 0) {  // prefix sums of the leaf counts
                int carry = 0;
                for (int b0 = 0; b0 < nl; b0 += 32) {
                    const int q = b0 + lane;
                    const int v = q < nl ? leafl[q].y : 0;
                    int inc = v;
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += y;
                    }
                    if (q < nl) lpre[q] = carry + inc - v;
                    carry += __shfl_sync(0xffffffffu, inc, 31);
                }
                if (lane == 0) lpre[nl] = carry;
            }
            __syncthreads();
            const int total = lpre[nl];
            for (int f0 = w * 32; f0 < total; f0 += KN_THREADS) {
                const int f = f0 + lane;
                bool in = false;
                float ox = 0.f, oy = 0.f, oz = 0.f;
                int j = 0;
                if (f < total) {
                    int lo = 0, hi = nl - 1;  // the last leaf starting at or before f
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (lpre[mid] <= f) lo = mid;
                        else hi = mid - 1;
                    }
                    j = leafl[lo].x + (f - lpre[lo]);
                    ox = grid_off(p.gcx[j], gref[0], p.grx[j], unit);
                    oy = grid_off(p.gcy[j], gref[1], p.gry[j], unit);
                    oz = grid_off(p.gcz[j], gref[2], p.grz[j], unit);
                    const float gx = fmaxf(0.f, fmaxf(blo[0] - ox, ox - bhi[0]));
                    const float gy = fmaxf(0.f, fmaxf(blo[1] - oy, oy - bhi[1]));
                    const float gz = fmaxf(0.f, fmaxf(blo[2] - oz, oz - bhi[2]));
                    in = gx * gx + gy * gy + gz * gz <= R2stage;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, in);
                if (bal == 0u) continue;
                int base = 0;
                if (lane == 0) base = atomicAdd(&S.nc, __popc(bal));
                base = __shfl_sync(0xffffffffu, base, 0);
                unsigned a2 = 0u;
                if (in) {
                    const int slot = base + __popc(bal & ltmask);
                    if (slot < KN_CAP) {
                        S.cand[slot] = make_float4(ox, oy, oz, __int_as_float(j));
                        a2 = __float_as_uint(ox * ox + oy * oy + oz * oz);
                    } else {
                        S.over = 1;
                    }
                }
                a2 = __reduce_max_sync(0xffffffffu, a2);
                if (lane == 0) atomicMax(&S.amax, a2);
            }
        }
        __syncthreads();
        const int nc = min(S.nc, KN_CAP);
        if (!S.over) {
            // group particles also bound the offsets
            for (int i = ga.x + tid; i < ga.x + ga.y; i += KN_THREADS) {
                float ox = grid_off(p.gcx[i], gref[0], p.grx[i], unit);
                float oy = grid_off(p.gcy[i], gref[1], p.gry[i], unit);
                float oz = grid_off(p.gcz[i], gref[2], p.grz[i], unit);
                atomicMax(&S.amax, __float_as_uint(ox * ox + oy * oy + oz * oz));
            }
            __syncthreads();
            // error bound of an FP32 d^2 near D (see the file comment)
            const float EA = 6.92820323f * (sqrtf(__uint_as_float(S.amax)) + 2.f * unit);  // 4 sqrt(3) A'
            const float R2 = R * R;
            const float thrR = R2 - 1.1920929e-07f * (EA * sqrtf(R2) + 5.f * R2);
            for (int i = ga.x + w; i < ga.x + ga.y; i += KN_WARPS) {
                const float xi = grid_off(p.gcx[i], gref[0], p.grx[i], unit);
                const float yi = grid_off(p.gcy[i], gref[1], p.gry[i], unit);
                const float zi = grid_off(p.gcz[i], gref[2], p.grz[i], unit);
                __syncwarp();  // the previous particle's scratch is no longer read
                if (lane == 0) { S.bn[w] = 0; S.un[w] = 0; }
                // bucket holding the 64th smallest; shrink this particle's
                // radius to that bucket while the bucket is too full to rank.
                // The first histogram pass also counts the candidates certainly
                // within R: fewer than n_ngb means the radius is too small.
                float R2i = R2, inv64 = 64.f / R2, R2sel = R2;
                int bstar = -1, kth = 0;
                bool ok = false, under_i = false;
                for (int it = 0; it < 16; it++) {
                    __syncwarp();
                    R2sel = R2i;  // the radius of this histogram (bstar, kth refer to it)
                    S.hist[w][lane] = 0;
                    S.hist[w][lane + 32] = 0;
                    __syncwarp();
                    inv64 = 64.f / R2i;
                    int cnt = 0;
                    for (int c = lane; c < nc; c += 32) {
                        float d = d2f(S.cand[c], xi, yi, zi);
                        if (it == 0) cnt += d <= thrR;
                        if (d <= R2i) atomicAdd(&S.hist[w][min(63, (int)(d * inv64))], 1);
                    }
                    if (it == 0 && warp_sum(cnt) < NGB) {
                        under_i = true;
                        break;
                    }
                    __syncwarp();
                    int h0 = S.hist[w][2 * lane], h1 = S.hist[w][2 * lane + 1];
                    int sum = h0 + h1, inc = sum;
                    for (int o = 1; o < 32; o <<= 1) {
                        int y = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += y;
                    }
                    int exc = inc - sum;
                    int mybin = -1, mybefore = 0;
                    if (exc < NGB && NGB <= exc + h0) { mybin = 2 * lane; mybefore = exc; }
                    else if (exc + h0 < NGB && NGB <= inc) { mybin = 2 * lane + 1; mybefore = exc + h0; }
                    unsigned bal = __ballot_sync(0xffffffffu, mybin >= 0);
                    if (bal == 0u) break;
                    int src = __ffs(bal) - 1;
                    bstar = __shfl_sync(0xffffffffu, mybin, src);
                    kth = NGB - __shfl_sync(0xffffffffu, mybefore, src);  // 1-based rank in bucket
                    if (S.hist[w][bstar] <= KN_BKT) { ok = true; break; }
                    R2i = R2i * (float)(bstar + 1) * (1.f / 64.f) * (1.f + 1e-6f);
                }
                if (under_i) {
                    if (lane == 0) S.under = 1;
                    continue;
                }
                float t = 0.f;
                bool have_t = false;
                if (ok) {
                    for (int c = lane; c < nc; c += 32) {
                        float d = d2f(S.cand[c], xi, yi, zi);
                        if (d <= R2i && min(63, (int)(d * inv64)) == bstar) {
                            int slot = atomicAdd(&S.bn[w], 1);
                            if (slot < KN_BKT) S.bkt[w][slot] = d;
                        }
                    }
                    __syncwarp();
                    const int nb = S.bn[w];
                    if (nb <= KN_BKT) {
                        // t = kth smallest value in the bucket (ties by position)
                        bool found = false;
                        for (int e = lane; e < nb; e += 32) {
                            float de = S.bkt[w][e];
                            int r = 0;
                            for (int f = 0; f < nb; f++) {
                                float df = S.bkt[w][f];
                                r += (df < de) || (df == de && f < e);
                            }
                            if (r == kth - 1) { t = de; found = true; }
                        }
                        unsigned fb = __ballot_sync(0xffffffffu, found);
                        if (fb != 0u) {
                            t = __shfl_sync(0xffffffffu, t, __ffs(fb) - 1);
                            have_t = true;
                        }
                    }
                }
                if (!have_t && bstar >= 0 && ga.y == 1) {
                    // a single particle whose bucket stays too full: exact
                    // selection over the candidates themselves (groups split
                    // first, which is cheaper for a clump inside a spread group)
                    bool okr = false;
                    t = knn_radix_kth(S, w, lane, nc, xi, yi, zi, R2sel, 64.f / R2sel, bstar, kth, &okr);
                    have_t = okr;
                }
                if (!have_t) {
                    if (lane == 0) knn_fail(S, ga.y, p.status);
                    continue;
                }
                // the bound at a point just above the band's upper end (E << t)
                const float tb = t * 1.0009765625f;
                const float E = 1.1920929e-07f * (EA * sqrtf(tb) + 5.f * tb);
                const float lo = t - 2.f * E, hi = t + 2.f * E;
                // classify: sure members written directly, uncertain ones collected
                int nS = 0;
                int *outn = p.nbr + (size_t)i * NGB;
                float *outd = p.nd2 + (size_t)i * NGB;
                for (int c0 = 0; c0 < nc; c0 += 32) {
                    int c = c0 + lane;
                    float d = 3.0e38f;
                    int j = -1;
                    if (c < nc) {
                        float4 cv = S.cand[c];
                        d = d2f(cv, xi, yi, zi);
                        j = __float_as_int(cv.w);
                    }
                    bool sure = d < lo;
                    unsigned sb = __ballot_sync(0xffffffffu, sure);
                    if (sure) {
                        int pos = nS + __popc(sb & ltmask);
                        if (pos < NGB) { outn[pos] = j; outd[pos] = d; }
                    }
                    nS += __popc(sb);
                    if (!sure && d <= hi) {
                        int slot = atomicAdd(&S.un[w], 1);
                        if (slot < KN_U) S.ui[w][slot] = j;
                    }
                }
                __syncwarp();
                const int nu = S.un[w];
                if (nu > KN_U || nS >= NGB) {
                    if (lane == 0) knn_fail(S, ga.y, p.status);
                    continue;
                }
                for (int e = lane; e < nu; e += 32) {
                    const int je = S.ui[w][e];
                    S.uD[w][e] = __double_as_longlong(exact_d2(p.gx, p.gy, p.gz, i, je));
                    S.ug[w][e] = p.ggrank[je];
                }
                __syncwarp();
                const int need = NGB - nS;
                double hsq = 0.0;
                int h64 = -1;
                bool have = false;
                for (int e = lane; e < nu; e += 32) {
                    const long long De = S.uD[w][e];
                    const int je = S.ui[w][e];
                    const int ge = S.ug[w][e];
                    int r = 0;
                    for (int f = 0; f < nu; f++) {  // integer compares: no FP64 work
                        const long long Df = S.uD[w][f];
                        r += (Df < De) || (Df == De && S.ug[w][f] < ge);
                    }
                    if (r < need) {
                        outn[nS + r] = je;
                        outd[nS + r] = (float)__longlong_as_double(De);
                    }
                    if (r == need - 1) { hsq = __longlong_as_double(De); h64 = ge; have = true; }
                }
                unsigned hb = __ballot_sync(0xffffffffu, have);
                if (hb == 0u) {  // error bound violated: fewer uncertain entries than needed
                    if (lane == 0) knn_fail(S, ga.y, p.status);
                    continue;
                }
                int hs = __ffs(hb) - 1;
                hsq = __shfl_sync(0xffffffffu, hsq, hs);
                h64 = __shfl_sync(0xffffffffu, h64, hs);
                __syncwarp();
                // density and EOS over the 64 neighbours
                const float hh = sqrtf((float)hsq);  // within one FP32 rounding of sqrt(h^2)
                const float hinv = 1.f / hh;
                float rs = 0.f, qs = 0.f;
                for (int e = lane; e < NGB; e += 32) {
                    int j = outn[e];
                    const float mw = p.gm[j] * kern_w(sqrtf(outd[e]), hinv);
                    rs += mw;
                    if (p.pressure) qs = __fmaf_rn(mw, p.gu[j], qs);
                }
                rs = warp_sum(rs);
                if (p.pressure) qs = warp_sum(qs);
                if (lane == 0) {
                    float u = p.gu[i];
                    float P = p.pressure ? (p.gamma - 1.f) * qs : (p.gamma - 1.f) * rs * u;
                    p.h2[i] = hsq;
                    p.h2lo[i] = __double2float_rd(hsq);
                    p.h2hi[i] = __double2float_ru(hsq);
                    p.h[i] = hh;
                    p.g64[i] = h64;
                    p.E[i] = E;
                    p.rho[i] = rs;
                    p.P[i] = P;
                    p.cs[i] = sqrtf(p.gamma * P / rs);
                }
            }
        }
        __syncthreads();
        if ((S.over || S.split) && ga.y > 1) {
            // the members need a radius whose candidates do not fit: hand
            // them to work items of at most KN_SUB consecutive particles
            // (single particles once the item is that small), each starting
            // from the margin x its members' largest previous support (at
            // most the group's radius); an item that still does not fit
            // splits again
            const int sub = ga.y > KN_SUB ? KN_SUB : 1;
            const int nsub = (ga.y + sub - 1) / sub;
            __syncthreads();
            if (tid == 0) {
                S.g = atomicAdd(p.nitems, nsub);
                S.wb = atomicAdd(p.nwl_out, nsub);
                p.kflag[gi] = 0;
                atomicAdd(p.remaining, 1);
            }
            __syncthreads();
            const int base = S.g;
            for (int k = tid; k < nsub; k += KN_THREADS) {
                const bool fits = base + k < p.item_cap;
                if (fits) {
                    const int f = ga.x + k * sub, cnt = min(sub, ga.y - k * sub);
                    p.item[base + k] = make_int2(f, cnt);
                    float hp = 0.f;
                    bool all = true;
                    for (int q = 0; q < cnt; q++) {
                        const float h = p.rprev[f + q];
                        hp = fmaxf(hp, h);
                        all = all && h > 0.f;
                    }
                    p.kR[base + k] = all ? fminf(R, p.margin * hp) : R;
                    p.kRb[base + k] = make_float2(0.f, 0.f);
                    p.kflag[base + k] = 1;
                } else {
                    atomicOr(p.status, ST_KNN_OVERFLOW);
                }
                // an item that did not fit is replaced by the finished parent
                if (S.wb + k < p.item_cap) p.wl_out[S.wb + k] = fits ? base + k : gi;
            }
            continue;
        }
        if (tid == 0) {
            float2 rb = p.kRb[gi];
            int done = 1;
            if (S.over) {
                rb.y = R;
                p.kR[gi] = rb.x > 0.f ? 0.5f * (R + rb.x) : 0.6f * R;
                done = 0;
            } else if (S.under) {
                rb.x = R;
                p.kR[gi] = rb.y > 0.f ? 0.5f * (R + rb.y) : 1.6f * R;
                done = 0;
                atomicAdd(p.nunder, 1);
            }
            p.kRb[gi] = rb;
            p.kflag[gi] = done ? 0 : 1;
            if (!done) {
                atomicAdd(p.remaining, 1);
                const int w = atomicAdd(p.nwl_out, 1);
                if (w < p.item_cap) p.wl_out[w] = gi;
            }
        }
    }
}

// ---------------------------------------------------------------- symmetric lists
// Bit k of mut[i] is set when entry k of N_i is mutual (i in N_j too), using
// (d^2, gas rank) <= (h_j^2, rank of j's n_ngb-th neighbour).  The FP32 d^2
// lies within 2 E_i of the FP64 one; the interval [d - 2E, d + 2E], widened
// by directed rounding, is first compared with h_j^2 rounded down and up to
// FP32 (no FP64 work: GB300 issues FP64 at a small fraction of the FP32
// rate).  Only a pair that test leaves open takes the FP64 test and, within
// its band, the exact FP64 d^2.  Every decision the FP32 test takes is the
// one the FP64 test would take.
__global__ void k_mutual(int ng, const int *__restrict__ nbr, const float *__restrict__ nd2,
                         const float *__restrict__ E, const double *__restrict__ h2, const float *__restrict__ h2lo,
                         const float *__restrict__ h2hi, const int *__restrict__ g64, const int *__restrict__ grank,
                         const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
                         unsigned long long *__restrict__ mut, int *__restrict__ rcnt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ng) return;
    unsigned long long mask = 0ull;
    const float Ei = E[i];
    const float e2 = 2.f * Ei;  // exact
    int gi = grank[i];
    for (int k = 0; k < NGB; k++) {
        int j = nbr[(size_t)i * NGB + k];
        if (j == i) { mask |= 1ull << k; continue; }
        const float df = nd2[(size_t)i * NGB + k];
        bool m;
        if (__fadd_ru(df, e2) < h2lo[j]) m = true;
        else if (__fsub_rd(df, e2) > h2hi[j]) m = false;
        else {
            double d = (double)df;
            double hj = h2[j];
            double e = 2.0 * (double)Ei;
            if (d + e < hj) m = true;
            else if (d - e > hj) m = false;
            else {
                double D = exact_d2(x, y, z, i, j);
                m = (D < hj) || (D == hj && gi <= g64[j]);
            }
        }
        if (m) mask |= 1ull << k;
        else atomicAdd(&rcnt[j], 1);
    }
    mut[i] = mask;
}

__global__ void k_rev_fill(int ng, const int *__restrict__ nbr, const unsigned long long *__restrict__ mut,
                           const int *__restrict__ roff, int *__restrict__ rfill, int *__restrict__ rlist)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ng) return;
    unsigned long long mask = mut[i];
    for (int k = 0; k < NGB; k++) {
        if (mask & (1ull << k)) continue;
        int j = nbr[(size_t)i * NGB + k];
        int s = atomicAdd(&rfill[j], 1);
        rlist[roff[j] + s] = i;
    }
}

// ---------------------------------------------------------------- force
struct ForceParams {
    int ng;
    const int *nbr, *roff, *rcnt, *rlist;
    const int4 *C;    // neighbour records (k_force_pack)
    const float4 *R, *V, *Q;
    const double *box;
    float alpha;
    float *ax, *ay, *az, *du;
    float *vsig;  // largest signal velocity c_i + c_j - 3 min(w_ij, 0) over the pairs of i
};

// One record set per gas particle so a pair gathers four records instead of
// fourteen fields: {cell, mass}, {residual, 1/h}, {v, c}, {rho, Y, U}.  The
// pressure terms of a pair are U_j Y_i gW(h_i) + U_i Y_j gW(h_j): Y = P/rho^2,
// U = 1 for density-energy SPH; Y = (gamma-1) u / P, U = (gamma-1) u for
// pressure-energy SPH with the smoothed P, whose pair coefficients are
// (gamma-1)^2 u_i u_j / P_i and / P_j.
__global__ void k_force_pack(int ng, const int *__restrict__ gcx, const int *__restrict__ gcy,
                             const int *__restrict__ gcz, const float *__restrict__ grx, const float *__restrict__ gry,
                             const float *__restrict__ grz, const float *__restrict__ gm, const float *__restrict__ gvx,
                             const float *__restrict__ gvy, const float *__restrict__ gvz, const float *__restrict__ h,
                             const float *__restrict__ rho, const float *__restrict__ P, const float *__restrict__ cs,
                             const float *__restrict__ gu, float gamma, int pressure, int4 *__restrict__ C,
                             float4 *__restrict__ R, float4 *__restrict__ V, float4 *__restrict__ Q)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ng) return;
    const float rj = rho[j];
    C[j] = make_int4(gcx[j], gcy[j], gcz[j], __float_as_int(gm[j]));
    R[j] = make_float4(grx[j], gry[j], grz[j], 1.f / h[j]);
    V[j] = make_float4(gvx[j], gvy[j], gvz[j], cs[j]);
    if (pressure) {
        const float U = (gamma - 1.f) * gu[j];
        Q[j] = make_float4(rj, U / P[j], U, 0.f);
    } else {
        Q[j] = make_float4(rj, P[j] / (rj * rj), 1.f, 0.f);
    }
}

__device__ __forceinline__ void pair_force(const ForceParams &p, int j, float unit, int ci0, int ci1, int ci2,
                                           float ri0, float ri1, float ri2, float vi0, float vi1, float vi2,
                                           float hinv_i, float pi_, float ui_, float rhoi, float csi, float &a0,
                                           float &a1, float &a2, float &du, float &vs)
{
    const int4 Cj = p.C[j];
    const float4 Rj = p.R[j];
    const float4 Vj = p.V[j];
    const float4 Qj = p.Q[j];
    float dx = __fmaf_rn((float)(ci0 - Cj.x), unit, ri0 - Rj.x);
    float dy = __fmaf_rn((float)(ci1 - Cj.y), unit, ri1 - Rj.y);
    float dz = __fmaf_rn((float)(ci2 - Cj.z), unit, ri2 - Rj.z);
    float r2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, dz * dz));
    float r = sqrtf(r2);
    float rinv = r > 0.f ? 1.f / r : 0.f;
    float dwi = kern_dw(r, hinv_i), dwj = kern_dw(r, Rj.w);
    float rhoj = Qj.x;
    float pj_ = Qj.y;
    float vx = vi0 - Vj.x, vy = vi1 - Vj.y, vz = vi2 - Vj.z;
    float w = (vx * dx + vy * dy + vz * dz) * rinv;
    float visc = 0.f;
    float vsig = csi + Vj.w - 3.f * fminf(w, 0.f);
    vs = fmaxf(vs, vsig);
    if (w < 0.f) visc = -0.5f * p.alpha * vsig * w / (0.5f * (rhoi + rhoj));
    float dwbar = 0.5f * (dwi + dwj);
    float mj = __int_as_float(Cj.w);
    const float ci = Qj.z * pi_, cj = ui_ * pj_;  // U_j Y_i, U_i Y_j
    float f = mj * (ci * dwi + cj * dwj + visc * dwbar) * rinv;
    a0 -= f * dx;
    a1 -= f * dy;
    a2 -= f * dz;
    du += mj * (ci * dwi + 0.5f * visc * dwbar) * w;
}

__global__ void k_force(ForceParams p)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.ng) return;
    const float unit = (float)p.box[4];
    const int4 Ci = p.C[i];
    const float4 Ri = p.R[i];
    const float4 Vi = p.V[i];
    const float4 Qi = p.Q[i];
    const int ci0 = Ci.x, ci1 = Ci.y, ci2 = Ci.z;
    const float ri0 = Ri.x, ri1 = Ri.y, ri2 = Ri.z;
    const float vi0 = Vi.x, vi1 = Vi.y, vi2 = Vi.z;
    const float hinv = Ri.w, rhoi = Qi.x, csi = Vi.w;
    const float pi_ = Qi.y, ui_ = Qi.z;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, du = 0.f, vs = 2.f * csi;
    const int *nb = p.nbr + (size_t)i * NGB;
    for (int k = 0; k < NGB; k++) {
        int j = nb[k];
        if (j == i) continue;
        pair_force(p, j, unit, ci0, ci1, ci2, ri0, ri1, ri2, vi0, vi1, vi2, hinv, pi_, ui_, rhoi, csi, a0, a1, a2, du,
                   vs);
    }
    int b = p.roff[i], e = b + p.rcnt[i];
    for (int k = b; k < e; k++)
        pair_force(p, p.rlist[k], unit, ci0, ci1, ci2, ri0, ri1, ri2, vi0, vi1, vi2, hinv, pi_, ui_, rhoi, csi, a0,
                   a1, a2, du, vs);
    p.ax[i] = a0;
    p.ay[i] = a1;
    p.az[i] = a2;
    p.du[i] = du;
    p.vsig[i] = vs;
}

// hydro results back to particle slots
__global__ void k_gas_scatter(int ng, const int *__restrict__ gslot, const float *__restrict__ hax,
                              const float *__restrict__ hay, const float *__restrict__ haz,
                              const float *__restrict__ hdu, float *__restrict__ ax, float *__restrict__ ay,
                              float *__restrict__ az, float *__restrict__ dudt)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ng) return;
    int s = gslot[k];
    ax[s] += hax[k];
    ay[s] += hay[k];
    az[s] += haz[k];
    dudt[s] = hdu[k];
}

__global__ void k_gas_scatter_density(int ng, const int *__restrict__ gslot, const float *__restrict__ grho,
                                      const float *__restrict__ gP, const float *__restrict__ gcs,
                                      const double *__restrict__ gh2, float *__restrict__ rho,
                                      float *__restrict__ pres, float *__restrict__ cs, double *__restrict__ h2)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ng) return;
    int s = gslot[k];
    rho[s] = grho[k];
    pres[s] = gP[k];
    cs[s] = gcs[k];
    h2[s] = gh2[k];
}

// ---------------------------------------------------------------- host
static int g_knn_blocks = 0;

int sph_density(gnb_ctx *c)
{
    int ng = (int)c->n_gas;
    if (ng == 0) return GNB_OK;
    phase_begin(c, GNB_T_HYDRO_TREE);
    PArr &a = c->P[c->cur];
    int gb = (ng + 255) / 256;
    // gas slots in Morton order
    GNB_TRY(gas_slots(c, a.type, c->n_d, c->gslot));
    GasGather gg;
    gg.skey = c->skey; gg.p = a; gg.gslot = c->gslot; gg.gkey = c->gkey;
    gg.gcx = c->gcx; gg.gcy = c->gcy; gg.gcz = c->gcz; gg.ggrank = c->ggrank;
    gg.grx = c->grx; gg.gry = c->gry; gg.grz = c->grz; gg.gm = c->gm;
    gg.gvx = c->gvx; gg.gvy = c->gvy; gg.gvz = c->gvz; gg.gu = c->gu; gg.gRprev = c->gRprev;
    gg.gx = c->gx; gg.gy = c->gy; gg.gz = c->gz;
    gg.ng = ng; gg.pred = c->use_pred ? 1 : 0; gg.have_h = c->have_h ? 1 : 0;
    gnb::counted(k_gas_gather)<<<gb, 256, 0, c->s>>>(gg);
    GNB_LAUNCH_CHECK(c, "gas gather");
    // hydro tree and groups of <= 32 gas particles (measured on the 2^24 disk
    // with the adaptive search margin: 7.05 ms for the kernel-size pass
    // against 7.12 with 24, 7.17 with 48 and 7.57 with 16; with the fixed
    // 1.1 margin 16 was best, since a wider radius makes a larger group's
    // candidates overflow)
    GNB_TRY(build_tree(c, c->gt, c->gkey, ng, c->ngas_d, c->cfg.n_leaf, 32, c->gcx, c->gcy, c->gcz, c->grx,
                       c->gry, c->grz, c->gm, c->gm, false));
    phase_begin(c, GNB_T_KNN);
    // work_d: [0] next item, [1] items left unfinished, [2] live item count, [3] per-pass snapshot
    gnb::counted(k_knn_init)<<<304, 256, 0, c->s>>>(c->gt, c->gRprev, c->have_h ? 1 : 0, c->knn_margin, c->box_d, c->kR,
                                      c->kRb, c->kflag, c->kitem, c->work_d + 2);
    GNB_LAUNCH_CHECK(c, "knn init");
    KnnParams p;
    p.na = c->gt.na; p.nb = c->gt.nb; p.item = c->kitem; p.nitems = c->work_d + 2; p.nsnap = c->work_d + 3;
    p.item_cap = (int)(2 * c->gcap + 1);
    p.gcx = c->gcx; p.gcy = c->gcy; p.gcz = c->gcz; p.ggrank = c->ggrank;
    p.grx = c->grx; p.gry = c->gry; p.grz = c->grz; p.gm = c->gm; p.gu = c->gu;
    p.gx = c->gx; p.gy = c->gy; p.gz = c->gz; p.box = c->box_d;
    p.kR = c->kR; p.kRb = c->kRb; p.kflag = c->kflag;
    p.rprev = c->gRprev;
    p.margin = c->knn_margin;
    p.nunder = c->work_d + 6;
    cudaMemsetAsync(c->work_d + 6, 0, sizeof(int), c->s);
    p.next = c->work_d; p.remaining = c->work_d + 1; p.status = c->status_d;
    p.nbr = c->nbr; p.nd2 = c->nd2; p.h2 = c->gh2; p.h2lo = c->gh2lo; p.h2hi = c->gh2hi; p.h = c->gh; p.E = c->gE; p.rho = c->grho; p.P = c->gP;
    p.cs = c->gcs; p.g64 = c->g64; p.gamma = (float)c->cfg.gamma; p.pressure = c->cfg.sph_variant;
    size_t smem = sizeof(KnnSmem);
    cudaError_t e = cudaFuncSetAttribute(k_knn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(c, e, "knn smem attribute");
    if (g_knn_blocks == 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_knn, KN_THREADS, smem);
        g_knn_blocks = sms * (per > 0 ? per : 1);
    }
    int passes = 0;
    const int rounds = 12;
    for (int round = 0; round < rounds; round++) {
        // four device passes per host check; each pass takes the worklist
        // the previous one wrote (the first takes every item)
        for (int q = 0; q < 4; q++) {
            const int o = passes & 1;
            cudaMemsetAsync(c->work_d, 0, 2 * sizeof(int), c->s);
            cudaMemsetAsync(c->work_d + 4 + o, 0, sizeof(int), c->s);
            if (passes == 0) {
                cudaMemcpyAsync(c->work_d + 3, c->work_d + 2, sizeof(int), cudaMemcpyDeviceToDevice, c->s);
                p.nsnap = c->work_d + 3;
                p.wl_in = nullptr;
            } else {
                p.nsnap = c->work_d + 4 + (o ^ 1);
                p.wl_in = c->kwl[o ^ 1];
            }
            p.wl_out = c->kwl[o];
            p.nwl_out = c->work_d + 4 + o;
            gnb::counted(k_knn)<<<g_knn_blocks, KN_THREADS, smem, c->s>>>(p);
            passes++;
        }
        GNB_LAUNCH_CHECK(c, "knn");
        cudaMemcpyAsync(c->pinned_i, c->work_d + 1, sizeof(int), cudaMemcpyDeviceToHost, c->s);
        cudaMemcpyAsync(c->pinned_i + 20, c->work_d + 3, sizeof(int), cudaMemcpyDeviceToHost, c->s);
        cudaMemcpyAsync(c->pinned_i + 21, c->work_d + 6, sizeof(int), cudaMemcpyDeviceToHost, c->s);
        cudaMemcpyAsync(c->pinned_i + 1, c->status_d, sizeof(int), cudaMemcpyDeviceToHost, c->s);
        GNB_TRY(cuda_check(c, cudaStreamSynchronize(c->s), "knn sync"));
        if (c->pinned_i[1] & ST_KNN_OVERFLOW) return fail(c, GNB_ECAPACITY, "kNN selection buffer overflow");
        if (c->pinned_i[0] == 0) break;
        if (round == rounds - 1) return fail(c, GNB_ECAPACITY, "kNN search radius did not converge");
    }
    c->stats[GNB_S_KNN_PASSES] = passes;
    // the next evaluation's margin: wider when more than 4 % of the work
    // items needed a larger radius, narrower (to 1.01) below 1 %.  On the
    // 2^24 disk (dt = 1e-3) a margin of 1.01 retries no item and takes
    // 7.57 ms for the pass, 1.05 7.83 ms, 1.1 8.21 ms; 1.0 retries 78 % of
    // the items (a support that did not shrink needs more than itself) and
    // takes 16.4 ms
    if (c->have_h) {
        const double under = (double)c->pinned_i[21] / (double)std::max(1, c->pinned_i[20]);
        if (under > 0.04) c->knn_margin = std::min(1.5f, c->knn_margin * 1.05f);
        else if (under < 0.01) c->knn_margin = std::max(1.01f, c->knn_margin / 1.02f);
    }
    c->stats[GNB_S_GAS_NODES] = c->gt.nnodes;
    gnb::counted(k_gas_scatter_density)<<<gb, 256, 0, c->s>>>(ng, c->gslot, c->grho, c->gP, c->gcs, c->gh2, c->rho, c->pres,
                                                c->cs, a.h2);
    GNB_LAUNCH_CHECK(c, "density scatter");
    phase_end(c);
    c->have_h = true;
    c->nbr_valid = true;
    return GNB_OK;
}

int sph_force(gnb_ctx *c)
{
    int ng = (int)c->n_gas;
    if (ng == 0) return GNB_OK;
    int gb = (ng + 255) / 256;
    phase_begin(c, GNB_T_FORCE);
    cudaMemsetAsync(c->rcnt, 0, sizeof(int) * ng, c->s);
    gnb::counted(k_mutual)<<<gb, 256, 0, c->s>>>(ng, c->nbr, c->nd2, c->gE, c->gh2, c->gh2lo, c->gh2hi, c->g64,
                                                 c->ggrank, c->gx, c->gy, c->gz, c->mut, c->rcnt);
    GNB_TRY(device_scan(c, c->rcnt, c->roff, c->ngas_d, ng, c->rtot_d));
    cudaMemsetAsync(c->rfill, 0, sizeof(int) * ng, c->s);
    gnb::counted(k_rev_fill)<<<gb, 256, 0, c->s>>>(ng, c->nbr, c->mut, c->roff, c->rfill, c->rlist);
    GNB_LAUNCH_CHECK(c, "symmetric lists");
    gnb::counted(k_force_pack)<<<gb, 256, 0, c->s>>>(ng, c->gcx, c->gcy, c->gcz, c->grx, c->gry, c->grz, c->gm, c->gvx,
                                                     c->gvy, c->gvz, c->gh, c->grho, c->gP, c->gcs, c->gu,
                                                     (float)c->cfg.gamma, c->cfg.sph_variant, c->fC, c->fR, c->fV,
                                                     c->fQ);
    ForceParams p;
    p.ng = ng; p.nbr = c->nbr; p.roff = c->roff; p.rcnt = c->rcnt; p.rlist = c->rlist;
    p.C = c->fC; p.R = c->fR; p.V = c->fV; p.Q = c->fQ;
    p.box = c->box_d; p.alpha = (float)c->cfg.alpha_visc;
    p.ax = c->hax; p.ay = c->hay; p.az = c->haz; p.du = c->hdu; p.vsig = c->gvsig;
    gnb::counted(k_force)<<<(ng + 127) / 128, 128, 0, c->s>>>(p);
    gnb::counted(k_gas_scatter)<<<gb, 256, 0, c->s>>>(ng, c->gslot, c->hax, c->hay, c->haz, c->hdu, c->ax, c->ay, c->az,
                                        c->dudt);
    GNB_LAUNCH_CHECK(c, "sph force");
    phase_end(c);
    return GNB_OK;
}

}  // namespace gnb
