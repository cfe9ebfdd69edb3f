// gravity.cu -- softened self-gravity (Eq. 1 of Hirashima et al., SC'25)
// by Barnes-Hut group walk (Sec. 3.4, 5.2.2, 5.2.4) or direct summation,
// plus the static NFW halo of the disk model.
//
// Design (GB300): one CTA of GW_THREADS threads per group, scheduled
// persistently from a device work counter.  The CTA walks the octree with a
// shared-memory stack, testing up to GW_THREADS cells at a time with the
// exact integer opening test, and stages accepted cells (monopole +
// quadrupole) and the particles of opened leaves in shared memory as FP32
// offsets from the group's reference grid point (Sec. 4.3 mixed precision).
// When a staging buffer fills, every thread evaluates its i-particle against
// the staged j entries, which are read as warp-wide broadcasts.  Small groups
// split the j loop over warps ("j-splits") so that all warps stay busy.
// Pair arithmetic is FP32 on the CUDA cores (not a dense contraction).
#include "common.cuh"

namespace gnb {

#define GW_THREADS 128
#define GW_STACK 4096
#define GW_LEAF 256
#define GW_JP 1024
#define GW_JC 256

struct GravParams {
    int4 *na, *nb;
    float4 *mo0, *mo1, *mo2;
    const int *groups, *ngroups;
    const int *cx, *cy, *cz;
    const float *rx, *ry, *rz, *m, *eps;
    float *ax, *ay, *az, *pot;
    const double *box;
    double theta2;
    float G;
    int quad;
    int n;
    int *next;
    int *status;
    unsigned long long *counters;
};

struct GravSmem {
    int stack[GW_STACK];
    int leaf[GW_LEAF];
    int leafoff[GW_LEAF + 1];
    float4 jp[GW_JP];
    float je[GW_JP];
    float4 c0[GW_JC], c1[GW_JC], c2[GW_JC];
    float4 red[GW_THREADS];
    int ws[32];
    int sp, nl, nc, g, bmin[3], bmax[3];
};

__device__ __forceinline__ bool must_open(int4 C, int level, const int *bmin, const int *bmax, double theta2)
{
    long long s = 1ll << (GNB_MAXLEV - level);
    bool overlap = true;
    long long d2 = 0;
    int cc[3] = {C.x, C.y, C.z};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        long long lo = cc[a], b0 = bmin[a], b1 = bmax[a];
        if (b0 > lo + s - 1 || b1 < lo) overlap = false;
        long long cen = 2 * lo + s;
        long long d = 0;
        if (2 * b0 > cen) d = 2 * b0 - cen;
        else if (cen > 2 * b1) d = cen - 2 * b1;
        d2 += d * d;
    }
    if (overlap) return true;
    double lhs = (double)(2 * s) * (double)(2 * s);
    return lhs > theta2 * (double)d2;
}

// Particle-particle: accumulate sum m_j (x_j - x_i)/R^3 and sum m_j/R, with
// R^2 = |x_j - x_i|^2 + eps_i^2 + eps_j^2.
template <bool MASK>
__device__ __forceinline__ void pp_loop(const GravSmem &S, int np, int split, int js, float xi, float yi, float zi,
                                        float e2i, float &ax, float &ay, float &az, float &ph)
{
#pragma unroll 4
    for (int j = split; j < np; j += js) {
        float4 q = S.jp[j];
        float e = S.je[j];
        float dx = q.x - xi, dy = q.y - yi, dz = q.z - zi;
        float r2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmaf_rn(dz, dz, e + e2i)));
        float ri = rsqrtf(r2);
        if (MASK) ri = r2 > 0.f ? ri : 0.f;
        float mr = q.w * ri;
        float mr3 = mr * ri * ri;
        ax = __fmaf_rn(mr3, dx, ax);
        ay = __fmaf_rn(mr3, dy, ay);
        az = __fmaf_rn(mr3, dz, az);
        ph += mr;
    }
}

// Particle-cell with monopole (+ traceless quadrupole), r = x_i - com:
//   a   += -M r/R^3 + Q r/R^5 - 5/2 (r.Q.r) r/R^7
//   phi += -M/R - 1/2 r.Q.r/R^5         (accumulated with the sign flipped)
template <bool QUAD>
__device__ __forceinline__ void pc_loop(const GravSmem &S, int nc, int split, int js, float xi, float yi, float zi,
                                        float e2i, float &ax, float &ay, float &az, float &ph)
{
#pragma unroll 2
    for (int c = split; c < nc; c += js) {
        float4 a = S.c0[c];
        float4 b = S.c1[c];
        float4 d = S.c2[c];
        float rx = xi - a.x, ry = yi - a.y, rz = zi - a.z;
        float R2 = __fmaf_rn(rx, rx, __fmaf_rn(ry, ry, __fmaf_rn(rz, rz, e2i + d.z)));
        float Ri = rsqrtf(R2);
        float Ri2 = Ri * Ri;
        float mR = a.w * Ri;
        float mR3 = mR * Ri2;
        if (QUAD) {
            float qx = __fmaf_rn(b.x, rx, __fmaf_rn(b.w, ry, d.x * rz));
            float qy = __fmaf_rn(b.w, rx, __fmaf_rn(b.y, ry, d.y * rz));
            float qz = __fmaf_rn(d.x, rx, __fmaf_rn(d.y, ry, b.z * rz));
            float rqr = __fmaf_rn(rx, qx, __fmaf_rn(ry, qy, rz * qz));
            float Ri5 = Ri2 * Ri2 * Ri;
            float Ri7 = Ri5 * Ri2;
            float t = 2.5f * rqr * Ri7 + mR3;
            ax += __fmaf_rn(qx, Ri5, -t * rx);
            ay += __fmaf_rn(qy, Ri5, -t * ry);
            az += __fmaf_rn(qz, Ri5, -t * rz);
            ph += __fmaf_rn(0.5f * rqr, Ri5, mR);
        } else {
            ax = __fmaf_rn(-mR3, rx, ax);
            ay = __fmaf_rn(-mR3, ry, ay);
            az = __fmaf_rn(-mR3, rz, az);
            ph += mR;
        }
    }
}

__device__ __forceinline__ int block_scan_excl(int v, int *ws, int *tot)
{
    int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = blockDim.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = lane < nw ? ws[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        ws[lane] = s;
    }
    __syncthreads();
    int r = x - v + (w > 0 ? ws[w - 1] : 0);
    *tot = ws[nw - 1];
    __syncthreads();
    return r;
}

template <bool MASK, bool QUAD>
__global__ void __launch_bounds__(GW_THREADS, 4) k_gravity_tree(GravParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GravSmem &S = *reinterpret_cast<GravSmem *>(smem_raw);
    const int tid = threadIdx.x;
    const float unit = (float)p.box[4];
    const int ngroups = *p.ngroups;
    unsigned long long cnt_pp = 0, cnt_pc = 0;

    for (;;) {
        if (tid == 0) S.g = atomicAdd(p.next, 1);
        __syncthreads();
        const int gi = S.g;
        if (gi >= ngroups) break;
        const int gnode = p.groups[gi];
        const int4 ga = p.na[gnode];
        const int gfirst = ga.x, gcount = ga.y;
        // bounding box of the whole group (its cells on the Morton grid)
        if (tid < 3) { S.bmin[tid] = 0x7fffffff; S.bmax[tid] = -1; }
        __syncthreads();
        for (int i = gfirst + tid; i < gfirst + gcount; i += GW_THREADS) {
            int cc[3] = {p.cx[i], p.cy[i], p.cz[i]};
#pragma unroll
            for (int a = 0; a < 3; a++) { atomicMin(&S.bmin[a], cc[a]); atomicMax(&S.bmax[a], cc[a]); }
        }
        __syncthreads();
        const int bmin[3] = {S.bmin[0], S.bmin[1], S.bmin[2]}, bmax[3] = {S.bmax[0], S.bmax[1], S.bmax[2]};
        const int gref[3] = {(bmin[0] + bmax[0]) >> 1, (bmin[1] + bmax[1]) >> 1, (bmin[2] + bmax[2]) >> 1};
        for (int i0 = 0; i0 < gcount; i0 += GW_THREADS) {
            const int icnt = min(GW_THREADS, gcount - i0);
            // j-splits: warps share i-particles and split the j loop
            // j-splits: each of the js = floor(128 / icnt) thread sets holds all
            // icnt i-particles and takes every js-th j entry
            const int ilanes = icnt;
            const int js = GW_THREADS / ilanes;
            const int islot = tid % ilanes, split = tid / ilanes;
            const bool ivalid = split < js;
            const int ip = gfirst + i0 + islot;
            const int ci[3] = {p.cx[ip], p.cy[ip], p.cz[ip]};
            const float xi = grid_off(ci[0], gref[0], p.rx[ip], unit);
            const float yi = grid_off(ci[1], gref[1], p.ry[ip], unit);
            const float zi = grid_off(ci[2], gref[2], p.rz[ip], unit);
            const float epi = p.eps[ip];
            const float e2i = epi * epi;
            float ax = 0.f, ay = 0.f, az = 0.f, ph = 0.f;
            if (tid == 0) { S.sp = 1; S.stack[0] = 0; S.nl = 0; S.nc = 0; }
            for (;;) {
                __syncthreads();
                const int sp = S.sp;
                const int nl0 = S.nl, nc0 = S.nc;
                // flush staged cells
                if (nc0 > GW_JC - GW_THREADS || (sp == 0 && nc0 > 0)) {
                    if (ivalid) pc_loop<QUAD>(S, nc0, split, js, xi, yi, zi, e2i, ax, ay, az, ph);
                    cnt_pc += (unsigned long long)nc0 * icnt;
                    __syncthreads();
                    if (tid == 0) S.nc = 0;
                }
                // flush pending leaves: expand to particles in chunks of GW_JP
                if (nl0 > GW_LEAF - GW_THREADS || (sp == 0 && nl0 > 0)) {
                    int total = 0;
                    for (int q0 = 0; q0 < nl0; q0 += GW_THREADS) {
                        int q = q0 + tid;
                        int v = q < nl0 ? p.na[S.leaf[q]].y : 0;
                        int tot;
                        int e = block_scan_excl(v, S.ws, &tot);
                        if (q < nl0) S.leafoff[q] = total + e;
                        total += tot;
                    }
                    if (tid == 0) S.leafoff[nl0] = total;
                    __syncthreads();
                    for (int c0 = 0; c0 < total; c0 += GW_JP) {
                        int np = min(GW_JP, total - c0);
                        for (int k = tid; k < np; k += GW_THREADS) {
                            int pos = c0 + k;
                            int lo = 0, hi = nl0 - 1;
                            while (lo < hi) {
                                int mid = (lo + hi + 1) >> 1;
                                if (S.leafoff[mid] <= pos) lo = mid;
                                else hi = mid - 1;
                            }
                            int j = p.na[S.leaf[lo]].x + (pos - S.leafoff[lo]);
                            float ej = p.eps[j];
                            S.jp[k] = make_float4(grid_off(p.cx[j], gref[0], p.rx[j], unit),
                                                  grid_off(p.cy[j], gref[1], p.ry[j], unit),
                                                  grid_off(p.cz[j], gref[2], p.rz[j], unit), p.m[j]);
                            S.je[k] = ej * ej;
                        }
                        __syncthreads();
                        if (ivalid) pp_loop<MASK>(S, np, split, js, xi, yi, zi, e2i, ax, ay, az, ph);
                        __syncthreads();
                    }
                    cnt_pp += (unsigned long long)total * icnt;
                    if (tid == 0) S.nl = 0;
                }
                __syncthreads();
                if (sp == 0) break;
                // pop k nodes; children pushed never exceed the stack
                int k = min(GW_THREADS, sp);
                int room = (GW_STACK - sp) / 7;
                if (room < 1) room = 1;
                k = min(k, room);
                int node = tid < k ? S.stack[sp - k + tid] : -1;
                __syncthreads();
                if (tid == 0) S.sp = sp - k;
                __syncthreads();
                if (node >= 0) {
                    int4 a = p.na[node];
                    int nch = a.w >> 8, lev = a.w & 255;
                    bool open = node == 0 || must_open(p.nb[node], lev, bmin, bmax, p.theta2);
                    if (!open) {
                        int slot = atomicAdd(&S.nc, 1);
                        int4 C = p.nb[node];
                        float4 m0 = p.mo0[node];
                        S.c0[slot] = make_float4(grid_off(C.x, gref[0], m0.x, unit), grid_off(C.y, gref[1], m0.y, unit),
                                                 grid_off(C.z, gref[2], m0.z, unit), m0.w);
                        S.c1[slot] = p.mo1[node];
                        S.c2[slot] = p.mo2[node];
                    } else if (nch == 0) {
                        int slot = atomicAdd(&S.nl, 1);
                        S.leaf[slot] = node;
                    } else {
                        int b = atomicAdd(&S.sp, nch);
                        if (b + nch <= GW_STACK) {
                            for (int q = 0; q < nch; q++) S.stack[b + q] = a.z + q;
                        } else {
                            atomicOr(p.status, ST_STACK_OVERFLOW);
                            atomicSub(&S.sp, nch);
                        }
                    }
                }
            }
            // reduce j-splits
            __syncthreads();
            S.red[tid] = make_float4(ax, ay, az, ph);
            __syncthreads();
            if (split == 0 && ivalid) {
                for (int s2 = 1; s2 < js; s2++) {
                    float4 r = S.red[tid + s2 * ilanes];
                    ax += r.x; ay += r.y; az += r.z; ph += r.w;
                }
                if (!MASK) ph -= p.m[ip] * rsqrtf(2.f * e2i);  // remove the j == i term
                p.ax[ip] = p.G * ax;
                p.ay[ip] = p.G * ay;
                p.az[ip] = p.G * az;
                p.pot[ip] = -p.G * ph;
            }
            __syncthreads();
        }
    }
    if (tid == 0) {
        atomicAdd(&p.counters[0], cnt_pp);
        atomicAdd(&p.counters[1], cnt_pc);
    }
}

// Direct summation: every group streams all n particles through shared memory.
template <bool MASK>
__global__ void __launch_bounds__(GW_THREADS, 4) k_gravity_direct(GravParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GravSmem &S = *reinterpret_cast<GravSmem *>(smem_raw);
    const int tid = threadIdx.x;
    const float unit = (float)p.box[4];
    const int ngroups = *p.ngroups;
    for (;;) {
        if (tid == 0) S.g = atomicAdd(p.next, 1);
        __syncthreads();
        const int gi = S.g;
        if (gi >= ngroups) break;
        const int4 ga = p.na[p.groups[gi]];
        for (int i0 = 0; i0 < ga.y; i0 += GW_THREADS) {
            const int icnt = min(GW_THREADS, ga.y - i0);
            const int ilanes = icnt;
            const int js = GW_THREADS / ilanes;
            const int islot = tid % ilanes, split = tid / ilanes;
            const bool ivalid = split < js;
            const int ip = ga.x + i0 + islot;
            const int gref[3] = {p.cx[ga.x + i0], p.cy[ga.x + i0], p.cz[ga.x + i0]};
            const float xi = grid_off(p.cx[ip], gref[0], p.rx[ip], unit);
            const float yi = grid_off(p.cy[ip], gref[1], p.ry[ip], unit);
            const float zi = grid_off(p.cz[ip], gref[2], p.rz[ip], unit);
            const float e2i = p.eps[ip] * p.eps[ip];
            float ax = 0.f, ay = 0.f, az = 0.f, ph = 0.f;
            for (int c0 = 0; c0 < p.n; c0 += GW_JP) {
                int np = min(GW_JP, p.n - c0);
                __syncthreads();
                for (int k = tid; k < np; k += GW_THREADS) {
                    int j = c0 + k;
                    float ej = p.eps[j];
                    S.jp[k] = make_float4(grid_off(p.cx[j], gref[0], p.rx[j], unit),
                                          grid_off(p.cy[j], gref[1], p.ry[j], unit),
                                          grid_off(p.cz[j], gref[2], p.rz[j], unit), p.m[j]);
                    S.je[k] = ej * ej;
                }
                __syncthreads();
                if (ivalid) pp_loop<MASK>(S, np, split, js, xi, yi, zi, e2i, ax, ay, az, ph);
            }
            __syncthreads();
            S.red[tid] = make_float4(ax, ay, az, ph);
            __syncthreads();
            if (split == 0 && ivalid) {
                for (int s2 = 1; s2 < js; s2++) {
                    float4 r = S.red[tid + s2 * ilanes];
                    ax += r.x; ay += r.y; az += r.z; ph += r.w;
                }
                if (!MASK) ph -= p.m[ip] * rsqrtf(2.f * e2i);
                p.ax[ip] = p.G * ax;
                p.ay[ip] = p.G * ay;
                p.az[ip] = p.G * az;
                p.pot[ip] = -p.G * ph;
            }
        }
        __syncthreads();
    }
}

static int g_sms = 0;

static GravParams make_params(gnb_ctx *c)
{
    PArr &a = c->P[c->cur];
    GravParams p;
    p.na = c->t.na; p.nb = c->t.nb; p.mo0 = c->t.mo0; p.mo1 = c->t.mo1; p.mo2 = c->t.mo2;
    p.groups = c->t.groups; p.ngroups = c->t.ngroups_d;
    p.cx = a.cx; p.cy = a.cy; p.cz = a.cz; p.rx = a.rx; p.ry = a.ry; p.rz = a.rz;
    p.m = a.m; p.eps = a.eps;
    p.ax = c->gax; p.ay = c->gay; p.az = c->gaz; p.pot = c->pot;
    p.box = c->box_d;
    p.theta2 = c->cfg.theta * c->cfg.theta;
    p.G = (float)c->cfg.G;
    p.quad = c->cfg.multipole;
    p.n = (int)c->n;
    p.next = c->pinned_i ? nullptr : nullptr;
    p.status = c->status_d;
    p.counters = c->counters_d;
    return p;
}

template <class K>
static int launch_persistent(gnb_ctx *c, K kern, GravParams p, int *next_d)
{
    size_t smem = sizeof(GravSmem);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(c, e, "gravity smem attribute");
    if (g_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, GW_THREADS, smem);
    if (per_sm < 1) per_sm = 1;
    p.next = next_d;
    cudaMemsetAsync(next_d, 0, sizeof(int), c->s);
    gnb::counted(kern)<<<g_sms * per_sm, GW_THREADS, smem, c->s>>>(p);
    GNB_LAUNCH_CHECK(c, "gravity kernel");
    return GNB_OK;
}

int gravity_tree(gnb_ctx *c)
{
    GravParams p = make_params(c);
    int *next_d = c->counters_d ? (int *)(c->counters_d + 6) : nullptr;
    bool q = c->cfg.multipole != 0;
    if (c->min_eps_zero) {
        if (q) return launch_persistent(c, k_gravity_tree<true, true>, p, next_d);
        return launch_persistent(c, k_gravity_tree<true, false>, p, next_d);
    }
    if (q) return launch_persistent(c, k_gravity_tree<false, true>, p, next_d);
    return launch_persistent(c, k_gravity_tree<false, false>, p, next_d);
}

int gravity_direct(gnb_ctx *c)
{
    GravParams p = make_params(c);
    int *next_d = (int *)(c->counters_d + 6);
    if (c->min_eps_zero) return launch_persistent(c, k_gravity_direct<true>, p, next_d);
    return launch_persistent(c, k_gravity_direct<false>, p, next_d);
}

// ---------------------------------------------------------------- NFW halo
// M(<r) = Ms [ln(1+r/rs) - (r/rs)/(1+r/rs)], a = -G M(<r) x / r^3,
// Phi = -G Ms ln(1 + r/rs) / r.
__global__ void k_nfw(const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
                      int n, float G, float ms, float rs, float *__restrict__ ax, float *__restrict__ ay,
                      float *__restrict__ az, float *__restrict__ pext)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float px = (float)x[i], py = (float)y[i], pz = (float)z[i];
    float r = sqrtf(px * px + py * py + pz * pz);
    float s = r / rs;
    float l1 = log1pf(s);
    float menc = ms * (l1 - s / (1.f + s));
    float f = r > 0.f ? -G * menc / (r * r * r) : 0.f;
    ax[i] = f * px;
    ay[i] = f * py;
    az[i] = f * pz;
    pext[i] = r > 0.f ? -G * ms * l1 / r : -G * ms / rs;
}

int gravity_nfw(gnb_ctx *c)
{
    int n = (int)c->n;
    PArr &a = c->P[c->cur];
    if (c->cfg.nfw_ms > 0) {
        gnb::counted(k_nfw)<<<(n + 255) / 256, 256, 0, c->s>>>(a.x, a.y, a.z, n, (float)c->cfg.G, (float)c->cfg.nfw_ms,
                                                 (float)c->cfg.nfw_rs, c->ax, c->ay, c->az, c->pext);
        GNB_LAUNCH_CHECK(c, "nfw");
    } else {
        cudaMemsetAsync(c->ax, 0, sizeof(float) * n, c->s);
        cudaMemsetAsync(c->ay, 0, sizeof(float) * n, c->s);
        cudaMemsetAsync(c->az, 0, sizeof(float) * n, c->s);
        cudaMemsetAsync(c->pext, 0, sizeof(float) * n, c->s);
    }
    return GNB_OK;
}

}  // namespace gnb
