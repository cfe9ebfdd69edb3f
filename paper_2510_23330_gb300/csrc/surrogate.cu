// surrogate.cu -- particle <-> grid mappings of the supernova surrogate and
// the batched surrogate step (Sec. 3.2-3.3 of Hirashima et al., SC'25): the
// gas in a (60 pc)^3 cube around each supernova is voxelised onto a 64^3 grid
// (SPH kernel convolution for the density, Shepard averages for temperature
// and velocity), the U-Net predicts the grid 0.1 Myr later, and the region's
// particles are replaced, keeping their IDs and number, by positions drawn
// from the predicted density with Gibbs sampling.
//
// Readings (the paper gives no formulas here):
//   channels  z0 = log10(max(rho, 1e-4)) + 0.33, z1 = (log10(max(T, 10)) - 2)/2,
//             z2..z4 = v / 20 (Msun/pc^3, K, km/s); empty voxels have rho = 0,
//             T = 10 K, v = 0; T = u * T_PER_U (mu = 0.6);
//   membership: a gas particle belongs to the first region whose cube
//             (|x - c|_inf <= side/2) contains it;
//   remap:   from the voxel of its old position, `sweeps` Gibbs sweeps over
//             x, y, z; each draw picks a voxel on the current line with
//             probability proportional to 10^(z0 - 0.33); FP64 CDF from index
//             0; then a uniform offset inside the voxel; draw k of particle
//             id uses U = (splitmix64(splitmix64(seed + id) + k) >> 11) 2^-53;
//             u and v are the predicted voxel's T / T_PER_U and 20 z.
#include <cuda_bf16.h>

#include "common.cuh"

typedef __nv_bfloat16 bf16;

namespace gnb {

int unet_prepare(gnb_unet *u, int batch, bf16 **xin, float **yout, int *grid, int *cout);
int unet_run(gnb_unet *u, int batch, cudaStream_t stream);

#define SUR_T_PER_U 48.45894937815476  // (gamma - 1) mu m_H / k_B, K per (km/s)^2, mu = 0.6

__device__ __forceinline__ uint64_t sm64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform01(uint64_t seed, uint64_t id, uint64_t k)
{
    return (double)(sm64(sm64(seed + id) + k) >> 11) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ float sur_w(float r, float hinv)
{
    float q = r * hinv;
    float s = 2.546479089470325f * hinv * hinv * hinv;
    if (q <= 0.5f) return s * (1.f - 6.f * q * q + 6.f * q * q * q);
    if (q <= 1.f) { float t = 1.f - q; return s * 2.f * t * t * t; }
    return 0.f;
}

// FP32 copy of the region centres for the membership pre-filter.
__global__ void k_centres_f32(const double *__restrict__ cent, int nreg, float *__restrict__ cf)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < 3 * nreg) cf[k] = (float)cent[k];
}

// Region of every gas particle: the first region r with |x - c_r|_inf <=
// side / 2, decided in FP64; an FP32 test with a margin far above its
// rounding error skips the regions that cannot contain the particle.
__global__ void k_region_assign(PArr p, int n, const double *__restrict__ cent, const float *__restrict__ cf, int nreg,
                                double half, int *__restrict__ reg, int *__restrict__ rcount)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int r = -1;
    if (p.type[i] == GNB_GAS) {
        double x = p.x[i], y = p.y[i], z = p.z[i];
        float xf = (float)x, yf = (float)y, zf = (float)z, hf = (float)half;
        for (int k = 0; k < nreg; k++) {
            float cx = cf[3 * k], cy = cf[3 * k + 1], cz = cf[3 * k + 2];
            float tol = hf + 1e-5f * (fabsf(xf) + fabsf(cx) + fabsf(yf) + fabsf(cy) + fabsf(zf) + fabsf(cz) + hf);
            if (fabsf(xf - cx) > tol || fabsf(yf - cy) > tol || fabsf(zf - cz) > tol) continue;
            if (fabs(x - cent[3 * k]) <= half && fabs(y - cent[3 * k + 1]) <= half && fabs(z - cent[3 * k + 2]) <= half) {
                r = k;
                break;
            }
        }
    }
    reg[i] = r;
    if (r >= 0) atomicAdd(&rcount[r], 1);
}

// Voxels whose centre can lie inside the kernel support of particle i
// (clipped to the grid): [i0, i1] per axis.
__device__ __forceinline__ void vox_footprint(const PArr &p, int i, const double *lo, double d, int grid, int *i0,
                                              int *i1)
{
    // explicit round-to-nearest operations: the counting and the filling pass
    // must derive the same tiles for a particle
    const double pp[3] = {p.x[i], p.y[i], p.z[i]};
    const double h = __dsqrt_rn(p.h2[i]);
    for (int a = 0; a < 3; a++) {
        i0[a] = max((int)floor(__dsub_rn(__ddiv_rn(__dsub_rn(__dsub_rn(pp[a], h), lo[a]), d), 0.5)), 0);
        i1[a] = min((int)ceil(__dsub_rn(__ddiv_rn(__dsub_rn(__dadd_rn(pp[a], h), lo[a]), d), 0.5)), grid - 1);
    }
}

__device__ __forceinline__ void region_lo(const double *cent, int r, double side, double *lo)
{
    for (int a = 0; a < 3; a++) lo[a] = cent[3 * r + a] - 0.5 * side;
}

// Voxelisation is binned by tiles of 8^3 voxels.  Pass 1: every member
// reserves one slot per tile its footprint touches (block-aggregated
// reservation against the list capacity) and counts itself into those tiles;
// a particle whose slots do not fit is flagged and goes through the direct
// scatter below instead.
__global__ void k_vox_bin_count(PArr p, int n, const int *__restrict__ reg, const double *__restrict__ cent,
                                double side, int grid, int tpa, unsigned long long cap,
                                unsigned long long *__restrict__ total, int *__restrict__ count,
                                unsigned char *__restrict__ ovf, int *__restrict__ any_ovf)
{
    __shared__ unsigned long long s_base;
    __shared__ unsigned s_sum;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int r = i < n ? reg[i] : -1;
    int i0[3] = {0, 0, 0}, i1[3] = {-1, -1, -1};
    unsigned np = 0;
    if (r >= 0) {
        double lo[3];
        region_lo(cent, r, side, lo);
        vox_footprint(p, i, lo, side / grid, grid, i0, i1);
        np = (unsigned)(((i1[0] >> 3) - (i0[0] >> 3) + 1) * ((i1[1] >> 3) - (i0[1] >> 3) + 1) *
                        ((i1[2] >> 3) - (i0[2] >> 3) + 1));
    }
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
    unsigned mine = np ? atomicAdd(&s_sum, np) : 0;
    __syncthreads();
    if (threadIdx.x == 0) s_base = s_sum ? atomicAdd(total, (unsigned long long)s_sum) : 0;
    __syncthreads();
    if (i >= n) return;
    if (r < 0) { ovf[i] = 0; return; }
    if (s_base + mine + np > cap) {
        ovf[i] = 1;
        *any_ovf = 1;
        return;
    }
    ovf[i] = 0;
    const int nt = tpa * tpa * tpa;
    int *cr = count + (size_t)r * nt;
    for (int tz = i0[2] >> 3; tz <= (i1[2] >> 3); tz++)
        for (int ty = i0[1] >> 3; ty <= (i1[1] >> 3); ty++)
            for (int tx = i0[0] >> 3; tx <= (i1[0] >> 3); tx++) atomicAdd(cr + (tz * tpa + ty) * tpa + tx, 1);
}

// Pass 2: write each member's index into the lists of its tiles.
__global__ void k_vox_bin_fill(PArr p, int n, const int *__restrict__ reg, const double *__restrict__ cent,
                               double side, int grid, int tpa, const unsigned char *__restrict__ ovf,
                               const int *__restrict__ off, const int *__restrict__ count, int *__restrict__ cur,
                               int *__restrict__ list)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int r = reg[i];
    if (r < 0 || ovf[i]) return;
    double lo[3];
    int i0[3], i1[3];
    region_lo(cent, r, side, lo);
    vox_footprint(p, i, lo, side / grid, grid, i0, i1);
    const size_t t0 = (size_t)r * tpa * tpa * tpa;
    for (int tz = i0[2] >> 3; tz <= (i1[2] >> 3); tz++)
        for (int ty = i0[1] >> 3; ty <= (i1[1] >> 3); ty++)
            for (int tx = i0[0] >> 3; tx <= (i1[0] >> 3); tx++) {
                size_t t = t0 + (tz * tpa + ty) * tpa + tx;
                int slot = atomicAdd(cur + t, 1);
                if (slot < count[t]) list[off[t] + slot] = i;  // never past the tile's counted slots
            }
}

// Direct scatter with global atomics, only for the particles flagged in pass 1
// acc[r][v][6] = {sum m W, sum (m/rho) W, sum T (m/rho) W, sum v (m/rho) W}
__global__ void k_vox_scatter(PArr p, int n, const int *__restrict__ reg, const unsigned char *__restrict__ ovf,
                              const float *__restrict__ rho, const double *__restrict__ cent, double side, int grid,
                              float *__restrict__ acc)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !ovf[i]) return;
    int r = reg[i];
    if (r < 0) return;
    double d = side / grid, lo[3];
    int i0[3], i1[3];
    region_lo(cent, r, side, lo);
    vox_footprint(p, i, lo, d, grid, i0, i1);
    float off[3] = {(float)(p.x[i] - lo[0]), (float)(p.y[i] - lo[1]), (float)(p.z[i] - lo[2])};
    float m = p.m[i], wr = m / rho[i];
    float T = p.u[i] * (float)SUR_T_PER_U;
    float vx = p.vx[i], vy = p.vy[i], vz = p.vz[i];
    float hinv = (float)(1.0 / sqrt(p.h2[i])), df = (float)d;
    float *base = acc + (size_t)r * grid * grid * grid * 6;
    for (int iz = i0[2]; iz <= i1[2]; iz++) {
        float dz = (iz + 0.5f) * df - off[2];
        for (int iy = i0[1]; iy <= i1[1]; iy++) {
            float dy = (iy + 0.5f) * df - off[1];
            for (int ix = i0[0]; ix <= i1[0]; ix++) {
                float dx = (ix + 0.5f) * df - off[0];
                float w = sur_w(sqrtf(dx * dx + dy * dy + dz * dz), hinv);
                if (w <= 0.f) continue;
                float *q = base + (((size_t)iz * grid + iy) * grid + ix) * 6;
                float ww = wr * w;
                atomicAdd(q + 0, m * w);
                atomicAdd(q + 1, ww);
                atomicAdd(q + 2, T * ww);
                atomicAdd(q + 3, vx * ww);
                atomicAdd(q + 4, vy * ww);
                atomicAdd(q + 5, vz * ww);
            }
        }
    }
}

// Pass 3: the tile lists are cut into chunks of at most VOX_CHUNK pairs so
// that a dense clump's tile is shared by many CTAs.  nchunk[t] chunks per
// tile; their exclusive scan gives each tile's first chunk.
#define VOX_CHUNK 1024
__global__ void k_vox_chunks(const int *__restrict__ count, const int *__restrict__ ntile_d, int *__restrict__ nchunk)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < *ntile_d) nchunk[t] = (count[t] + VOX_CHUNK - 1) / VOX_CHUNK;
}

// Persistent CTAs over chunks, gather form (no shared-memory atomics): the
// 8 warps own the 8 z-slices of the tile and each lane owns two voxels of its
// slice, (x, y) = (lane % 8, lane / 8) and (lane % 8, lane / 8 + 4), with
// their six sums in registers.  The chunk's particles are staged in shared
// memory 256 at a time; every warp reads each staged particle by broadcast,
// skips it when its footprint misses the warp's slice, and otherwise adds
// the kernel weight at its two voxel centres.  Sums are added to the global
// accumulators acc[r][v][6] once per chunk.
struct VoxP {
    float ox, oy, oz, h2, hinv, m, wr, T, vx, vy, vz;
    int zlo, zhi;
};

__global__ void __launch_bounds__(256) k_vox_tile(PArr p, const float *__restrict__ rho,
                                                  const double *__restrict__ cent, double side, int grid, int tpa,
                                                  const int *__restrict__ ntile_d, const int *__restrict__ off,
                                                  const int *__restrict__ cnt, const int *__restrict__ choff,
                                                  const int *__restrict__ nchunks_d, const int *__restrict__ list,
                                                  float *__restrict__ vacc)
{
    __shared__ VoxP sp[256];
    const int nt = tpa * tpa * tpa, ntile = *ntile_d, nchunks = *nchunks_d;
    const double d = side / grid;
    const float df = (float)d;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t G = (size_t)grid;
    for (int cid = blockIdx.x; cid < nchunks; cid += gridDim.x) {
        int lo_t = 0, hi_t = ntile;  // last tile whose first chunk is <= cid
        while (lo_t < hi_t) {
            int mid = (lo_t + hi_t) >> 1;
            if (choff[mid] <= cid) lo_t = mid + 1;
            else hi_t = mid;
        }
        const int tile = lo_t - 1;
        const int r = tile / nt, t = tile % nt;
        const int x0 = 8 * (t % tpa), y0 = 8 * ((t / tpa) % tpa), z0 = 8 * (t / (tpa * tpa));
        const int k = cid - choff[tile];
        const int beg = off[tile] + k * VOX_CHUNK, end = off[tile] + min(cnt[tile], (k + 1) * VOX_CHUNK);
        double lo[3];
        region_lo(cent, r, side, lo);
        const int iz = z0 + warp, ix = x0 + (lane & 7), iy0 = y0 + (lane >> 3), iy1 = iy0 + 4;
        const float cx = (ix + 0.5f) * df, cy0 = (iy0 + 0.5f) * df, cy1 = (iy1 + 0.5f) * df, cz = (iz + 0.5f) * df;
        float a0[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, a1[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int b = beg; b < end; b += 256) {
            __syncthreads();  // the previous batch has been read by every warp
            const int q = b + threadIdx.x;
            if (q < end) {
                const int i = list[q];
                int i0[3], i1[3];
                vox_footprint(p, i, lo, d, grid, i0, i1);
                VoxP v;
                v.ox = (float)(p.x[i] - lo[0]);
                v.oy = (float)(p.y[i] - lo[1]);
                v.oz = (float)(p.z[i] - lo[2]);
                const double h = sqrt(p.h2[i]);
                v.hinv = (float)(1.0 / h);
                v.h2 = 1.f / (v.hinv * v.hinv);
                v.m = p.m[i];
                v.wr = v.m / rho[i];
                v.T = p.u[i] * (float)SUR_T_PER_U;
                v.vx = p.vx[i]; v.vy = p.vy[i]; v.vz = p.vz[i];
                v.zlo = i0[2];
                v.zhi = i1[2];
                sp[threadIdx.x] = v;
            }
            __syncthreads();
            const int nb = min(256, end - b);
            for (int j = 0; j < nb; j++) {
                const VoxP &v = sp[j];
                if (iz < v.zlo || iz > v.zhi) continue;  // warp-uniform
                const float dz = cz - v.oz, dx = cx - v.ox;
                const float dxz = dx * dx + dz * dz;
                const float dy0 = cy0 - v.oy, dy1 = cy1 - v.oy;
                const float r20 = dxz + dy0 * dy0, r21 = dxz + dy1 * dy1;
                if (r20 < v.h2) {
                    const float w = sur_w(sqrtf(r20), v.hinv);
                    const float ww = v.wr * w;
                    a0[0] += v.m * w; a0[1] += ww; a0[2] += v.T * ww;
                    a0[3] += v.vx * ww; a0[4] += v.vy * ww; a0[5] += v.vz * ww;
                }
                if (r21 < v.h2) {
                    const float w = sur_w(sqrtf(r21), v.hinv);
                    const float ww = v.wr * w;
                    a1[0] += v.m * w; a1[1] += ww; a1[2] += v.T * ww;
                    a1[3] += v.vx * ww; a1[4] += v.vy * ww; a1[5] += v.vz * ww;
                }
            }
        }
        if (ix < grid && iz < grid) {
            const size_t rb = (size_t)r * G * G * G;
            if (iy0 < grid) {
                float *g = vacc + (rb + ((size_t)iz * G + iy0) * G + ix) * 6;
                for (int c = 0; c < 6; c++)
                    if (a0[c] != 0.f) atomicAdd(g + c, a0[c]);
            }
            if (iy1 < grid) {
                float *g = vacc + (rb + ((size_t)iz * G + iy1) * G + ix) * 6;
                for (int c = 0; c < 6; c++)
                    if (a1[c] != 0.f) atomicAdd(g + c, a1[c]);
            }
        }
    }
}

// standardised channels; FP32 [r][v][5] and/or BF16 [r][2][v][8] (the U-Net's
// input: 16 channels blocked by 8, vs voxels per region)
__global__ void k_vox_finalize(const float *__restrict__ acc, long long nv, long long vs, float *__restrict__ out,
                               bf16 *__restrict__ outb)
{
    long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const float *a = acc + v * 6;
    float rho_v = a[0], den = a[1];
    float T = den > 0.f ? a[2] / den : 10.f;
    float z[5];
    z[0] = log10f(fmaxf(rho_v, 1e-4f)) + 0.33f;
    z[1] = (log10f(fmaxf(T, 10.f)) - 2.f) * 0.5f;
    for (int c = 0; c < 3; c++) z[2 + c] = den > 0.f ? a[3 + c] / den / 20.f : 0.f;
    if (out)
        for (int c = 0; c < 5; c++) out[v * 5 + c] = z[c];
    if (outb) {
        long long r = v / vs, sv = v - r * vs;
        bf16 *b0 = outb + (r * 2 * vs + sv) * 8;
        for (int c = 0; c < 8; c++) b0[c] = __float2bfloat16_rn(c < 5 ? z[c] : 0.f);
        bf16 *b1 = b0 + vs * 8;
        for (int c = 0; c < 8; c++) b1[c] = __float2bfloat16_rn(0.f);
    }
}

__global__ void k_set_int(int *p, int v) { *p = v; }

static int vox_sms()
{
    static int n = []() {
        int d = 0, v = 0;
        cudaGetDevice(&d);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d);
        return v > 0 ? v : 1;
    }();
    return n;
}

__global__ void k_remap_weights(const float *__restrict__ pred, long long nv, int cout, double *__restrict__ w)
{
    long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < nv) w[v] = pow(10.0, (double)pred[v * cout] - 0.33);
}

// Cumulative weights along every grid line of every region, one thread per
// (region, axis, line), summed left to right in FP64 -- the same additions in
// the same order as a running sum taken at draw time, so each draw below sees
// bit-identical partial sums.  Line of axis a through voxel (x, y, z):
// a = 0 -> z G + y, a = 1 -> z G + x, a = 2 -> y G + x.
__global__ void k_line_cdf(const double *__restrict__ w, int nreg, int grid, double *__restrict__ cdf)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long G = grid, lines = G * G;
    if (t >= (long long)nreg * 3 * lines) return;
    const long long line = t % lines, ra = t / lines;
    const int a = (int)(ra % 3);
    const long long r = ra / 3;
    const long long u = line / G, v = line % G;  // the two fixed coordinates (outer, inner)
    long long b0, stride;
    if (a == 0) { b0 = (u * G + v) * G; stride = 1; }          // z = u, y = v
    else if (a == 1) { b0 = u * G * G + v; stride = G; }       // z = u, x = v
    else { b0 = u * G + v; stride = G * G; }                   // y = u, x = v
    const double *wr = w + r * G * G * G + b0;
    double *out = cdf + t * G;
    double cum = 0.0;
    for (int q = 0; q < grid; q++) {
        cum = __dadd_rn(cum, wr[q * stride]);
        out[q] = cum;
    }
}

__global__ void k_remap(PArr p, int n, const int *__restrict__ reg, const float *__restrict__ pred, int cout,
                        const double *__restrict__ cdf, const double *__restrict__ cent, double side, int grid,
                        const unsigned long long *__restrict__ seedp, int sweeps)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int r = reg[i];
    if (r < 0) return;
    uint64_t seed = *seedp;
    double d = side / grid;
    double lo[3] = {cent[3 * r] - 0.5 * side, cent[3 * r + 1] - 0.5 * side, cent[3 * r + 2] - 0.5 * side};
    double pp[3] = {p.x[i], p.y[i], p.z[i]};
    int c[3];
    for (int a = 0; a < 3; a++) {
        double f = floor(__ddiv_rn(__dsub_rn(pp[a], lo[a]), d));
        c[a] = f < 0.0 ? 0 : (f > (double)(grid - 1) ? grid - 1 : (int)f);
    }
    const size_t G = (size_t)grid;
    uint64_t id = (uint64_t)p.id[i];
    uint64_t k = 0;
    for (int s = 0; s < sweeps; s++) {
        for (int a = 0; a < 3; a++, k++) {
            // the line through the current voxel along axis a; pick the first
            // q whose running sum exceeds U * total (binary search of the
            // non-decreasing running sums = the first crossing of a scan)
            size_t line = a == 0 ? (size_t)c[2] * G + c[1] : (a == 1 ? (size_t)c[2] * G + c[0] : (size_t)c[1] * G + c[0]);
            const double *L = cdf + (((size_t)r * 3 + a) * G * G + line) * G;
            double target = __dmul_rn(uniform01(seed, id, k), L[grid - 1]);
            int qa = 0, qb = grid;
            while (qa < qb) {
                int mid = (qa + qb) >> 1;
                if (L[mid] > target) qb = mid;
                else qa = mid + 1;
            }
            c[a] = qa < grid ? qa : grid - 1;
        }
    }
    double np[3];
    for (int a = 0; a < 3; a++) np[a] = lo[a] + (c[a] + uniform01(seed, id, (uint64_t)(3 * sweeps + a))) * d;
    p.x[i] = np[0];
    p.y[i] = np[1];
    p.z[i] = np[2];
    const float *pv = pred + ((((size_t)r * grid + c[2]) * grid + c[1]) * grid + c[0]) * cout;
    double T = pow(10.0, 2.0 * (double)pv[1] + 2.0);
    p.u[i] = (float)(T / SUR_T_PER_U);
    p.vx[i] = 20.f * pv[2];
    p.vy[i] = 20.f * pv[3];
    p.vz[i] = 20.f * pv[4];
}

// ---------------------------------------------------------------- host
int voxelise_buffers_for(gnb_ctx *c, int nreg, int grid)
{
    size_t nv = (size_t)nreg * grid * grid * grid;
    if (c->sur_pcap < c->cap) {
        c->sur_gen++;
        dfree(c, c->sreg); dfree(c, c->vovf);
        c->sreg = nullptr; c->vovf = nullptr;
        GNB_TRY(dalloc(c, &c->sreg, (size_t)c->cap + 1));
        GNB_TRY(dalloc(c, &c->vovf, (size_t)c->cap + 1));
        c->sur_pcap = c->cap;
    }
    if (c->sur_nv < nv || c->sur_nreg < nreg) {
        c->sur_gen++;
        dfree(c, c->vacc); dfree(c, c->vw); dfree(c, c->vcdf); dfree(c, c->cent_d); dfree(c, c->rcount);
        dfree(c, c->vout); dfree(c, c->centf);
        c->vacc = nullptr; c->vw = nullptr; c->vcdf = nullptr; c->cent_d = nullptr; c->rcount = nullptr;
        c->vout = nullptr; c->centf = nullptr;
        GNB_TRY(dalloc(c, &c->vacc, nv * 6));
        GNB_TRY(dalloc(c, &c->vw, nv));
        GNB_TRY(dalloc(c, &c->vcdf, nv * 3));
        GNB_TRY(dalloc(c, &c->vout, nv * 5));
        GNB_TRY(dalloc(c, &c->cent_d, (size_t)nreg * 3));
        GNB_TRY(dalloc(c, &c->centf, (size_t)nreg * 3));
        GNB_TRY(dalloc(c, &c->rcount, (size_t)nreg));
        c->sur_nv = nv;
        c->sur_nreg = nreg;
    }
    const size_t tpa = (size_t)(grid + 7) / 8, ntile = (size_t)nreg * tpa * tpa * tpa;
    if (c->vt_ntile < ntile) {
        c->sur_gen++;
        dfree(c, c->vt_count); dfree(c, c->vt_off); dfree(c, c->vt_cur); dfree(c, c->vt_choff);
        c->vt_count = nullptr; c->vt_off = nullptr; c->vt_cur = nullptr; c->vt_choff = nullptr;
        GNB_TRY(dalloc(c, &c->vt_count, ntile));
        GNB_TRY(dalloc(c, &c->vt_off, ntile + 1));
        GNB_TRY(dalloc(c, &c->vt_cur, ntile));
        GNB_TRY(dalloc(c, &c->vt_choff, ntile + 1));
        c->vt_ntile = ntile;
    }
    // tile-list slots: a support of h reaches about 2 h / 8 voxels + 1 tiles per
    // axis; six per particle covers the usual supports, the rest overflow to
    // the direct scatter
    const size_t lcap = 6 * (size_t)c->cap + ((size_t)1 << 20);
    if (c->vt_cap < lcap) {
        c->sur_gen++;
        dfree(c, c->vt_list);
        c->vt_list = nullptr;
        GNB_TRY(dalloc(c, &c->vt_list, lcap));
        c->vt_cap = lcap;
    }
    if (!c->vt_total) GNB_TRY(dalloc(c, &c->vt_total, 1));
    if (!c->vt_misc) GNB_TRY(dalloc(c, &c->vt_misc, 4));
    if (!c->seed_d) GNB_TRY(dalloc(c, &c->seed_d, 1));
    return GNB_OK;
}

// Region membership and accumulators; the finalised channels go to `out`
// (FP32 [nreg][grid^3][5]) and/or `outb` (BF16 U-Net input).
static int vox_launch(gnb_ctx *c, int nreg, double side, int grid, float *out, bf16 *outb)
{
    int n = (int)c->n;
    PArr &a = c->P[c->cur];
    size_t nv = (size_t)nreg * grid * grid * grid;
    const int tpa = (grid + 7) / 8;
    const long long ntile = (long long)nreg * tpa * tpa * tpa;
    cudaMemsetAsync(c->rcount, 0, sizeof(int) * nreg, c->s);
    counted(k_centres_f32)<<<(3 * nreg + 255) / 256, 256, 0, c->s>>>(c->cent_d, nreg, c->centf);
    counted(k_region_assign)<<<(n + 255) / 256, 256, 0, c->s>>>(a, n, c->cent_d, c->centf, nreg, 0.5 * side,
                                                                c->sreg, c->rcount);
    cudaMemsetAsync(c->vacc, 0, sizeof(float) * nv * 6, c->s);
    cudaMemsetAsync(c->vt_count, 0, sizeof(int) * ntile, c->s);
    cudaMemsetAsync(c->vt_cur, 0, sizeof(int) * ntile, c->s);
    cudaMemsetAsync(c->vt_total, 0, sizeof(unsigned long long), c->s);
    cudaMemsetAsync(c->vt_misc, 0, 4 * sizeof(int), c->s);
    counted(k_set_int)<<<1, 1, 0, c->s>>>(c->vt_misc, (int)ntile);
    counted(k_vox_bin_count)<<<(n + 255) / 256, 256, 0, c->s>>>(a, n, c->sreg, c->cent_d, side, grid, tpa,
                                                                (unsigned long long)c->vt_cap, c->vt_total,
                                                                c->vt_count, c->vovf, c->vt_misc + 1);
    GNB_TRY(device_scan(c, c->vt_count, c->vt_off, c->vt_misc, (int)ntile, nullptr));
    counted(k_vox_bin_fill)<<<(n + 255) / 256, 256, 0, c->s>>>(a, n, c->sreg, c->cent_d, side, grid, tpa, c->vovf,
                                                               c->vt_off, c->vt_count, c->vt_cur, c->vt_list);
    counted(k_vox_scatter)<<<(n + 127) / 128, 128, 0, c->s>>>(a, n, c->sreg, c->vovf, c->rho, c->cent_d, side, grid,
                                                              c->vacc);
    counted(k_vox_chunks)<<<(unsigned)((ntile + 255) / 256), 256, 0, c->s>>>(c->vt_count, c->vt_misc, c->vt_cur);
    GNB_TRY(device_scan(c, c->vt_cur, c->vt_choff, c->vt_misc, (int)ntile, c->vt_misc + 2));
    counted(k_vox_tile)<<<(unsigned)(vox_sms() * 8), 256, 0, c->s>>>(
        a, c->rho, c->cent_d, side, grid, tpa, c->vt_misc, c->vt_off, c->vt_count, c->vt_choff, c->vt_misc + 2,
        c->vt_list, c->vacc);
    counted(k_vox_finalize)<<<(unsigned)((nv + 255) / 256), 256, 0, c->s>>>(
        c->vacc, (long long)nv, (long long)grid * grid * grid, out, outb);
    GNB_LAUNCH_CHECK(c, "voxelise");
    return GNB_OK;
}

static int remap_launch(gnb_ctx *c, int nreg, double side, int grid, const float *pred, int cout, int sweeps)
{
    int n = (int)c->n;
    size_t nv = (size_t)nreg * grid * grid * grid;
    counted(k_remap_weights)<<<(unsigned)((nv + 255) / 256), 256, 0, c->s>>>(pred, (long long)nv, cout, c->vw);
    long long nl = (long long)nreg * 3 * grid * grid;
    counted(k_line_cdf)<<<(unsigned)((nl + 127) / 128), 128, 0, c->s>>>(c->vw, nreg, grid, c->vcdf);
    counted(k_remap)<<<(n + 127) / 128, 128, 0, c->s>>>(c->P[c->cur], n, c->sreg, pred, cout, c->vcdf, c->cent_d,
                                                        side, grid, c->seed_d, sweeps);
    GNB_LAUNCH_CHECK(c, "remap");
    return GNB_OK;
}

int voxelise(gnb_ctx *c, int nreg, const double *centers, double side, int grid, float *out_dev)
{
    GNB_TRY(voxelise_buffers_for(c, nreg, grid));
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(c->cent_d, centers, sizeof(double) * 3 * nreg, cudaMemcpyHostToDevice,
                                          c->s), "centres"));
    phase_begin(c, GNB_T_VOXELISE);
    int rc = vox_launch(c, nreg, side, grid, out_dev ? out_dev : c->vout, nullptr);
    phase_end(c);
    return rc;
}

int remap_regions(gnb_ctx *c, int nreg, const double *centers, double side, int grid, const float *pred_dev,
                  uint64_t seed, int sweeps)
{
    GNB_TRY(voxelise_buffers_for(c, nreg, grid));
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(c->cent_d, centers, sizeof(double) * 3 * nreg, cudaMemcpyHostToDevice,
                                          c->s), "centres"));
    unsigned long long sd = seed;
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(c->seed_d, &sd, sizeof(sd), cudaMemcpyHostToDevice, c->s), "seed"));
    int n = (int)c->n;
    cudaMemsetAsync(c->rcount, 0, sizeof(int) * nreg, c->s);
    counted(k_centres_f32)<<<(3 * nreg + 255) / 256, 256, 0, c->s>>>(c->cent_d, nreg, c->centf);
    counted(k_region_assign)<<<(n + 255) / 256, 256, 0, c->s>>>(c->P[c->cur], n, c->cent_d, c->centf, nreg, 0.5 * side,
                                                                c->sreg, c->rcount);
    phase_begin(c, GNB_T_REMAP);
    GNB_TRY(remap_launch(c, nreg, side, grid, pred_dev, 5, sweeps));
    phase_end(c);
    return cuda_check(c, cudaStreamSynchronize(c->s), "remap sync");
}

// voxelise -> U-Net -> remap for nreg regions; after the first call with a
// given shape the whole sequence is replayed as one CUDA graph.
int sn_surrogate_batch(gnb_ctx *c, gnb_unet *net, int nreg, const double *centers, double side, uint64_t seed,
                       int sweeps, int use_graph)
{
    bf16 *xin = nullptr;
    float *yout = nullptr;
    int grid = 0, cout = 0;
    GNB_TRY(unet_prepare(net, nreg, &xin, &yout, &grid, &cout));
    if (cout != 5) return fail(c, GNB_EINVAL, "the surrogate network must predict 5 channels");
    GNB_TRY(voxelise_buffers_for(c, nreg, grid));
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(c->cent_d, centers, sizeof(double) * 3 * nreg, cudaMemcpyHostToDevice,
                                          c->s), "centres"));
    unsigned long long sd = seed;
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(c->seed_d, &sd, sizeof(sd), cudaMemcpyHostToDevice, c->s), "seed"));
    bool same = c->sn_graph && c->sn_key[0] == nreg && c->sn_key[1] == grid && c->sn_key[2] == sweeps &&
                c->sn_net == (void *)net && c->sn_side == side && c->sn_n == c->n && c->sn_cur == c->cur &&
                c->sn_gen == c->sur_gen;
    if (use_graph && same) {
        c->sn_graph_replays++;
        return cuda_check(c, cudaGraphLaunch(c->sn_graph, c->s), "surrogate graph launch");
    }
    auto issue = [&]() -> int {
        phase_begin(c, GNB_T_VOXELISE);
        GNB_TRY(vox_launch(c, nreg, side, grid, nullptr, xin));
        phase_begin(c, GNB_T_UNET);
        GNB_TRY(unet_run(net, nreg, c->s));
        phase_begin(c, GNB_T_REMAP);
        int rc = remap_launch(c, nreg, side, grid, yout, cout, sweeps);
        phase_end(c);
        return rc;
    };
    // with the phase timers on, the batch runs eagerly (no graph) so that
    // each stage's events are recorded
    if (!use_graph || c->s == nullptr || c->timing) return issue();
    if (c->sn_graph) {
        cudaGraphExecDestroy(c->sn_graph);
        c->sn_graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    GNB_TRY(cuda_check(c, cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal), "begin capture"));
    int rc = issue();
    cudaError_t e = cudaStreamEndCapture(c->s, &g);
    if (rc != GNB_OK) { if (g) cudaGraphDestroy(g); return rc; }
    GNB_TRY(cuda_check(c, e, "end capture"));
    e = cudaGraphInstantiate(&c->sn_graph, g, 0);
    cudaGraphDestroy(g);
    GNB_TRY(cuda_check(c, e, "graph instantiate"));
    c->sn_key[0] = nreg; c->sn_key[1] = grid; c->sn_key[2] = sweeps;
    c->sn_net = net; c->sn_side = side; c->sn_n = c->n; c->sn_cur = c->cur; c->sn_gen = c->sur_gen;
    return cuda_check(c, cudaGraphLaunch(c->sn_graph, c->s), "surrogate graph launch");
}

}  // namespace gnb
