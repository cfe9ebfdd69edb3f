// sn.cu -- supernova energy injection and the CFL timestep of the plain
// (small-timestep) integration of a supernova region (Sec. 1: the CFL
// condition makes the timestep tiny around supernovae; Sec. 3.2-3.3: the
// conventional integration the surrogate replaces and is trained on).
//
// Injection (a reading; the paper gives only the 10^51 erg energy, Sec. 1):
// thermal energy E goes to the n_ngb gas particles nearest to the explosion
// point, ordered by (FP64 d^2, gas rank) like the kernel-size search, with
// weights W(r_j, h) of the cubic spline whose support h is the distance to
// the n_ngb-th of them; du_j = E W_j / (m_j sum_k W_k).  The weights, their
// sum and the energy added are FP64.
//
// CFL (a reading of Sec. 1's condition): dt = C min_i h_i / vsig_i with
// vsig_i = max_j (c_i + c_j - 3 min(w_ij, 0)) over the symmetric neighbours.
#include "common.cuh"

namespace gnb {

#define SN_THREADS 1024

__device__ __forceinline__ double sn_w(double r, double h)
{
    double q = r / h, s = 8.0 / (3.141592653589793 * h * h * h);
    if (q <= 0.5) return s * (1.0 - 6.0 * q * q + 6.0 * q * q * q);
    if (q <= 1.0) { double t = 1.0 - q; return s * 2.0 * t * t * t; }
    return 0.0;
}

__device__ __forceinline__ double sn_d2(double px, double py, double pz, double x, double y, double z)
{
    double dx = __dsub_rn(x, px), dy = __dsub_rn(y, py), dz = __dsub_rn(z, pz);
    double a = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    return __dadd_rn(a, __dmul_rn(dz, dz));
}

template <class T>
__device__ __forceinline__ T block_sum(T v, T *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    T s = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); q++) s += sh[q];
    return s;
}

// One block: select the k nearest gas particles of (px, py, pz) by bitwise
// search on the FP64 d^2 pattern (non-negative doubles order like their bit
// patterns), ties by gas rank, then add the kernel-weighted energy.
// out = {sum of weights, energy added, h, number heated}.
__global__ void __launch_bounds__(SN_THREADS) k_inject(PArr p, int n, double px, double py, double pz, double E,
                                                       int k, double *out)
{
    __shared__ long long shl[32];
    __shared__ double shd[32];
    auto count_lt = [&](unsigned long long T, int rank_lim, bool use_rank) -> long long {
        long long c = 0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            if (p.type[i] != GNB_GAS) continue;
            unsigned long long b = (unsigned long long)__double_as_longlong(sn_d2(px, py, pz, p.x[i], p.y[i], p.z[i]));
            if (!use_rank) c += b < T;
            else c += (b == T && p.grank[i] < rank_lim);
        }
        return block_sum<long long>(c, shl);
    };
    unsigned long long D = 0;
    for (int b = 62; b >= 0; b--) {
        unsigned long long cand = D | (1ull << b);
        if (count_lt(cand, 0, false) < k) D = cand;
    }
    long long below = count_lt(D, 0, false);   // strictly closer than the k-th distance
    long long need = k - below;                // taken from the ties at distance D, lowest ranks
    int R = 0;
    for (int b = 30; b >= 0; b--) {
        int cand = R | (1 << b);
        if (count_lt(D, cand, true) < need) R = cand;
    }
    // members: d2 < D, or d2 == D and rank <= R
    double h = sqrt(__longlong_as_double((long long)D));
    double ws = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (p.type[i] != GNB_GAS) continue;
        double d2 = sn_d2(px, py, pz, p.x[i], p.y[i], p.z[i]);
        unsigned long long b = (unsigned long long)__double_as_longlong(d2);
        if (b < D || (b == D && p.grank[i] <= R)) ws += h > 0.0 ? sn_w(sqrt(d2), h) : 1.0;
    }
    ws = block_sum<double>(ws, shd);
    double added = 0.0;
    long long heated = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (p.type[i] != GNB_GAS) continue;
        double d2 = sn_d2(px, py, pz, p.x[i], p.y[i], p.z[i]);
        unsigned long long b = (unsigned long long)__double_as_longlong(d2);
        if (b < D || (b == D && p.grank[i] <= R)) {
            double wj = h > 0.0 ? sn_w(sqrt(d2), h) : 1.0;
            double du = E * wj / ((double)p.m[i] * ws);
            float u0 = p.u[i];
            float u1 = (float)((double)u0 + du);
            p.u[i] = u1;
            added += (double)p.m[i] * ((double)u1 - (double)u0);
            heated++;
        }
    }
    added = block_sum<double>(added, shd);
    heated = block_sum<long long>(heated, shl);
    if (threadIdx.x == 0) {
        out[0] = ws;
        out[1] = added;
        out[2] = h;
        out[3] = (double)heated;
    }
}

int inject_energy(gnb_ctx *c, const double pos[3], double E, double out[4])
{
    counted(k_inject)<<<1, SN_THREADS, 0, c->s>>>(c->P[c->cur], (int)c->n, pos[0], pos[1], pos[2], E,
                                                 c->cfg.n_ngb, c->red_d);
    GNB_LAUNCH_CHECK(c, "inject");
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(out, c->red_d, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->s),
                       "inject copy"));
    return cuda_check(c, cudaStreamSynchronize(c->s), "inject sync");
}

// min over gas of h_i / vsig_i (two levels: block partials, then one block)
__global__ void k_cfl_partial(const float *__restrict__ h, const float *__restrict__ vsig, int ng,
                              double *__restrict__ part)
{
    __shared__ double sh[32];
    double m = 1e300;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ng; i += gridDim.x * blockDim.x) {
        double v = (double)vsig[i];
        double t = v > 0.0 ? (double)h[i] / v : 1e300;
        m = t < m ? t : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        double q = __shfl_xor_sync(0xffffffffu, m, o);
        m = q < m ? q : m;
    }
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = sh[0];
        for (int q = 1; q < (int)(blockDim.x >> 5); q++) r = sh[q] < r ? sh[q] : r;
        part[blockIdx.x] = r;
    }
}

__global__ void k_cfl_final(const double *__restrict__ part, int nb, double *__restrict__ out)
{
    if (threadIdx.x != 0) return;
    double r = 1e300;
    for (int b = 0; b < nb; b++) r = part[b] < r ? part[b] : r;
    out[0] = r;
}

int cfl_min_h_over_vsig(gnb_ctx *c, double *out)
{
    int ng = (int)c->n_gas;
    if (ng == 0) {
        *out = 1e300;
        return GNB_OK;
    }
    int nb = 256;
    counted(k_cfl_partial)<<<nb, 256, 0, c->s>>>(c->gh, c->gvsig, ng, c->red_d);
    counted(k_cfl_final)<<<1, 32, 0, c->s>>>(c->red_d, nb, c->red_d + 256);
    GNB_LAUNCH_CHECK(c, "cfl");
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(out, c->red_d + 256, sizeof(double), cudaMemcpyDeviceToHost, c->s),
                       "cfl copy"));
    return cuda_check(c, cudaStreamSynchronize(c->s), "cfl sync");
}

}  // namespace gnb
