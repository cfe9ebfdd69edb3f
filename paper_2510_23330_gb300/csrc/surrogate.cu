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

#include <algorithm>

#include "common.cuh"

typedef __nv_bfloat16 bf16;

namespace gnb {

int unet_prepare(gnb_unet *u, int batch, bf16 **xin, float **yout, int *grid, int *cout);
int unet_run(gnb_unet *u, int batch, cudaStream_t stream, const bf16 *xin, float *yout);

#define SUR_T_PER_U 48.45894937815476  // (gamma - 1) mu m_H / k_B, K per (km/s)^2, mu = 0.6

__device__ __forceinline__ uint64_t sm64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Draw k of a particle whose stream is sid = splitmix64(seed + id): a uniform
// double in [0, 1) from the top 53 bits of splitmix64(sid + k).
__device__ __forceinline__ double uniform_draw(uint64_t sid, uint64_t k)
{
    return (double)(sm64(sid + k) >> 11) * (1.0 / 9007199254740992.0);
}

// counter[key] += 1 for every active lane, one atomic per distinct key in
// the warp (neighbouring particles in Morton order mostly share their
// region and tiles); returns each lane's slot.
__device__ __forceinline__ int warp_inc(int *counter, int key)
{
    const unsigned mask = __match_any_sync(__activemask(), key);
    const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(counter + key, __popc(mask));
    base = __shfl_sync(mask, base, leader);
    return base + __popc(mask & ((1u << lane) - 1));
}

// Region of every gas particle: the first region r (smallest index) with
// |x - c_r|_inf <= side / 2, decided in FP64.  Candidates come from the
// regions sorted by centre x: an FP32 binary search finds the slab
// |c_x - x| <= half and an FP32 test on all three axes filters it, both with
// a margin far above the FP32 rounding of the coordinates; only the
// survivors get the exact FP64 test (GB300's FP64 rate is a small fraction
// of its FP32 rate).
__global__ void k_region_assign(PArr p, int n, const double *__restrict__ cent, const float *__restrict__ rsx,
                                const int *__restrict__ rsi, const float *__restrict__ cf, int nreg, double half,
                                int *__restrict__ reg, int *__restrict__ rcount)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int r = -1;
    if (p.type[i] == GNB_GAS) {
        const double x = p.x[i], y = p.y[i], z = p.z[i];
        const float xf = (float)x, yf = (float)y, zf = (float)z, hf = (float)half;
        const float tol = 1e-5f * (fabsf(xf) + fabsf(yf) + fabsf(zf) + hf) + 1e-30f;
        const float xl = xf - hf - tol, xr = xf + hf + tol;
        int a = 0, b = nreg;
        while (a < b) {
            int m = (a + b) >> 1;
            if (rsx[m] < xl) a = m + 1;
            else b = m;
        }
        int best = nreg;
        for (int k = a; k < nreg && rsx[k] <= xr; k++) {
            const int q = rsi[k];
            if (q >= best) continue;
            const float tq = tol + 1e-5f * (fabsf(cf[3 * q]) + fabsf(cf[3 * q + 1]) + fabsf(cf[3 * q + 2]));
            if (fabsf(yf - cf[3 * q + 1]) > hf + tq || fabsf(zf - cf[3 * q + 2]) > hf + tq) continue;
            if (fabs(x - cent[3 * q]) <= half && fabs(y - cent[3 * q + 1]) <= half && fabs(z - cent[3 * q + 2]) <= half)
                best = q;
        }
        if (best < nreg) r = best;
    }
    reg[i] = r;
    if (r >= 0) warp_inc(rcount, r);
}

__device__ __forceinline__ void region_lo(const double *cent, int r, double side, double *lo)
{
    for (int a = 0; a < 3; a++) lo[a] = cent[3 * r + a] - 0.5 * side;
}

// Voxelisation, pass 1: every region member's FP32 values are computed once
// and staged as three float4 -- offset from the region corner (the one FP64
// step: the difference of two FP64 positions) and h^2; 1/h, m s, (m/rho) s,
// T; velocity and the packed z range of the footprint (s = 8 / (pi h^3), the
// kernel normalisation) -- plus the packed x and y ranges (grids of at most
// 256 voxels per axis).  The footprint box only bounds the walk of pass 2,
// which tests every voxel exactly, so it is taken in FP32 and widened by one
// voxel on each side.
__global__ void k_vox_stage(PArr p, int n, const int *__restrict__ reg, int r0, int r1, const float *__restrict__ rho,
                            const double *__restrict__ cent, double side, int grid, float4 *__restrict__ vpa,
                            float4 *__restrict__ vpb, float4 *__restrict__ vpc, int *__restrict__ vbox)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int r = reg[i];
    if (r < r0 || r >= r1) return;  // not a member of regions [r0, r1)
    double lo[3];
    region_lo(cent, r, side, lo);
    const float rel[3] = {(float)(p.x[i] - lo[0]), (float)(p.y[i] - lo[1]), (float)(p.z[i] - lo[2])};
    const float h2 = (float)p.h2[i], h = sqrtf(h2), hinv = 1.f / h;
    const float idf = (float)grid / (float)side;
    int i0[3], i1[3];
    for (int a = 0; a < 3; a++) {
        i0[a] = max((int)floorf((rel[a] - h) * idf - 0.5f) - 1, 0);
        i1[a] = min((int)ceilf((rel[a] + h) * idf - 0.5f) + 1, grid - 1);
    }
    const float sn = 2.546479089470325f * hinv * hinv * hinv;  // 8 / (pi h^3)
    const float m = p.m[i];
    vpa[i] = make_float4(rel[0], rel[1], rel[2], h2);
    vpb[i] = make_float4(hinv, m * sn, m / rho[i] * sn, p.u[i] * (float)SUR_T_PER_U);
    vpc[i] = make_float4(p.vx[i], p.vy[i], p.vz[i], __int_as_float((i0[2] << 16) | i1[2]));
    vbox[i] = i0[0] | (i1[0] << 8) | (i0[1] << 16) | (i1[1] << 24);
}

__device__ __forceinline__ float m4_shape(float q)
{
    // cubic spline without its normalisation: 1 - 6q^2 + 6q^3 (q <= 1/2),
    // 2 (1 - q)^3 (1/2 < q <= 1), 0 beyond
    if (q <= 0.5f) return 1.f - 6.f * q * q + 6.f * q * q * q;
    if (q <= 1.f) { float t = 1.f - q; return 2.f * t * t * t; }
    return 0.f;
}

// Pass 2, one thread per member particle: the six kernel-weighted terms
// {m W, (m/rho) W, T (m/rho) W, v (m/rho) W} of every voxel inside the
// particle's support are added with vector reductions resolved at L2: the
// first four to accA[r][v][4] (red.global.add.v4.f32), the last two to
// accB[r][v / 2][4], which holds them for the voxel pair (2u, 2u + 1) side
// by side, so that two neighbouring voxels of a row take one v4 reduction
// (a voxel without its partner, one v2).  One reduction costs one L2
// operation at any width, and the pass is bound by their number: 1.5 per
// deposit instead of 2.  The thread walks the (y, z) rows of the footprint
// box and, in each row, only the x-range that can lie inside the support
// (conservatively wide; the exact r^2 test decides), so only voxels near the
// support sphere are visited.  Neighbouring threads take neighbouring
// particles (Morton order): their smoothing lengths and footprints are
// alike, so the lanes of a warp run loops of similar length, and their
// reductions hit voxels that are close in memory.  No FP64 arithmetic runs
// here.
__device__ __forceinline__ void red_v4(float *a, float x, float y, float z, float w)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"l"(a), "f"(x), "f"(y), "f"(z), "f"(w)
                 : "memory");
}
__device__ __forceinline__ void red_v2(float *a, float x, float y)
{
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};\n" ::"l"(a), "f"(x), "f"(y) : "memory");
}

__global__ void __launch_bounds__(256) k_vox_scatter(int n, const int *__restrict__ reg, int r0, int r1,
                                                     const float4 *__restrict__ vpa, const float4 *__restrict__ vpb,
                                                     const float4 *__restrict__ vpc, const int *__restrict__ vbox,
                                                     double side, int grid, float *__restrict__ accA,
                                                     float *__restrict__ accB)
{
    // members of regions [r0, r1); accA and accB hold those regions
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int r = reg[i];
    if (r < r0 || r >= r1) return;
    const float df = (float)(side / grid), idf = 1.f / df;
    const size_t G = (size_t)grid;
    const float4 pa = vpa[i], pb = vpb[i], pc = vpc[i];
    const int bx = vbox[i], bz = __float_as_int(pc.w);
    const int x0 = bx & 0xff, x1 = (bx >> 8) & 0xff, y0 = (bx >> 16) & 0xff, y1 = (bx >> 24) & 0xff;
    const int z0 = bz >> 16, z1 = bz & 0xffff;
    const size_t vbase = (size_t)(r - r0) * G * G * G;
    for (int iz = z0; iz <= z1; iz++) {
        const float dz = (iz + 0.5f) * df - pa.z;
        for (int iy = y0; iy <= y1; iy++) {
            const float dy = (iy + 0.5f) * df - pa.y;
            const float dyz2 = dy * dy + dz * dz;
            const float rem = pa.w - dyz2;
            if (rem <= 0.f) continue;
            const float sx = sqrtf(rem);
            const int lo = max(x0, (int)floorf((pa.x - sx) * idf - 0.5f));
            const int hi = min(x1, (int)ceilf((pa.x + sx) * idf - 0.5f));
            const size_t vrow = vbase + ((size_t)iz * G + iy) * G;
            // (vy, vz) terms of an even voxel wait for their odd partner
            bool pend = false;
            float p4 = 0.f, p5 = 0.f;
            for (int ix = lo; ix <= hi; ix++) {
                const size_t v = vrow + ix;
                const float dx = (ix + 0.5f) * df - pa.x;
                const float r2 = dx * dx + dyz2;
                float w = 0.f;
                if (r2 < pa.w) w = m4_shape(sqrtf(r2) * pb.x);
                const bool dep = w > 0.f;
                const float ww = pb.z * w;
                if (dep) red_v4(accA + v * 4, pb.y * w, ww, pb.w * ww, pc.x * ww);
                float *qb = accB + (v >> 1) * 4;
                if ((v & 1) == 0) {
                    if (dep) {
                        if (ix == hi) red_v2(qb, pc.y * ww, pc.z * ww);
                        else { pend = true; p4 = pc.y * ww; p5 = pc.z * ww; }
                    }
                } else {
                    if (pend && dep) red_v4(qb, p4, p5, pc.y * ww, pc.z * ww);
                    else if (pend) red_v2(qb, p4, p5);
                    else if (dep) red_v2(qb + 2, pc.y * ww, pc.z * ww);
                    pend = false;
                }
            }
        }
    }
}

// standardised channels; FP32 [r][v][5] and/or BF16 [r][2][v][8] (the U-Net's
// input: 16 channels blocked by 8, vs voxels per region).  blockIdx.y is the
// region; each voxel's sums are read as two float4 and its eight BF16
// channels of each block stored as one 16-byte word.
__global__ void __launch_bounds__(256) k_vox_finalize(const float *__restrict__ accA, const float *__restrict__ accB,
                                                     size_t v0, int vs, float *__restrict__ out,
                                                     bf16 *__restrict__ outb)
{
    const int sv = blockIdx.x * blockDim.x + threadIdx.x;
    if (sv >= vs) return;
    const size_t r = blockIdx.y, v = r * (size_t)vs + sv, va = v0 + v;  // va: index in the accumulators
    const float4 a0 = reinterpret_cast<const float4 *>(accA)[va];
    const float2 a1 = reinterpret_cast<const float2 *>(accB)[(va >> 1) * 2 + (va & 1)];
    const float rho_v = a0.x, den = a0.y;
    const float T = den > 0.f ? a0.z / den : 10.f;
    float z[5];
    z[0] = log10f(fmaxf(rho_v, 1e-4f)) + 0.33f;
    z[1] = (log10f(fmaxf(T, 10.f)) - 2.f) * 0.5f;
    z[2] = den > 0.f ? a0.w / den / 20.f : 0.f;
    z[3] = den > 0.f ? a1.x / den / 20.f : 0.f;
    z[4] = den > 0.f ? a1.y / den / 20.f : 0.f;
    if (out)
        for (int c = 0; c < 5; c++) out[v * 5 + c] = z[c];
    if (outb) {
        __nv_bfloat162 h[4] = {__floats2bfloat162_rn(z[0], z[1]), __floats2bfloat162_rn(z[2], z[3]),
                               __floats2bfloat162_rn(z[4], 0.f), __floats2bfloat162_rn(0.f, 0.f)};
        uint4 *b0 = reinterpret_cast<uint4 *>(outb + (r * 2 * vs + sv) * 8);
        *b0 = *reinterpret_cast<const uint4 *>(h);
        b0[vs] = make_uint4(0u, 0u, 0u, 0u);  // channels 8..15 of the block layout
    }
}

__global__ void k_remap_weights(const float *__restrict__ pred, long long nv, int cout, double *__restrict__ w)
{
    long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < nv) w[v] = exp10((double)pred[v * cout] - 0.33);
}

// Cumulative weights along every grid line of every region, one thread per
// (region, axis, line), summed left to right in FP64 -- the same additions in
// the same order as a running sum taken at draw time, so each draw below sees
// bit-identical partial sums -- and each sum also rounded to nearest FP32;
// every 8th FP32 sum also goes to a coarse table (grids of a multiple of 8).  Line of axis a through voxel (x, y, z):
// a = 0 -> z G + y, a = 1 -> z G + x, a = 2 -> y G + x.
__global__ void k_line_cdf(const double *__restrict__ w, int nreg, int grid, double *__restrict__ cdf,
                           float *__restrict__ cdf32, float *__restrict__ cdfc)
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
    float *out32 = cdf32 + t * G;
    double cum = 0.0;
    for (int q = 0; q < grid; q++) {
        cum = __dadd_rn(cum, wr[q * stride]);
        out[q] = cum;
        out32[q] = __double2float_rn(cum);
        if ((grid & 7) == 0 && (q & 7) == 7) cdfc[t * (G >> 3) + (q >> 3)] = out32[q];
    }
}

// The same sums for grids of 32 or 64 voxels per axis, one warp per 32
// consecutive lines (same region and axis) staged through shared memory:
// the weights are read and the sums written as contiguous blocks (a line of
// axis 0 is contiguous; lines of axes 1 and 2 are read across the warp),
// and each lane sums its own line left to right as above (bit-identical).
constexpr int LC_W = 2;  // warps per block
__global__ void __launch_bounds__(32 * LC_W) k_line_cdf_tiled(const double *__restrict__ w, int nreg, int grid,
                                                              double *__restrict__ cdf, float *__restrict__ cdf32,
                                                              float *__restrict__ cdfc)
{
    __shared__ double tile[LC_W][32][65];
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const long long G = grid, lines = G * G;
    const long long t0 = ((long long)blockIdx.x * LC_W + wq) * 32;  // first line of this warp
    if (t0 >= (long long)nreg * 3 * lines) return;                  // (warp-uniform)
    const long long line0 = t0 % lines, ra = t0 / lines;
    const int a = (int)(ra % 3);
    const long long r = ra / 3;
    const long long u = line0 / G, v0 = line0 % G;
    const double *wr = w + r * G * G * G;
    double(*T)[65] = tile[wq];
    if (a == 0) {
        // lines (z = u, y = v0 .. v0 + 31) along x: one contiguous block of 32 G weights
        const double *blk = wr + (u * G + v0) * G;
        for (int k = lane; k < 32 * grid; k += 32) T[k / grid][k % grid] = blk[k];
    } else {
        const long long stride = a == 1 ? G : G * G;
        const long long b0 = a == 1 ? u * G * G + v0 : u * G + v0;  // line l adds l (inner x)
        for (int q = 0; q < grid; q++) T[lane][q] = wr[b0 + lane + q * stride];
    }
    __syncwarp();
    double cum = 0.0;
    for (int q = 0; q < grid; q++) {
        cum = __dadd_rn(cum, T[lane][q]);
        T[lane][q] = cum;
    }
    __syncwarp();
    double *out = cdf + t0 * G;
    float *out32 = cdf32 + t0 * G;
    for (int k = lane; k < 32 * grid; k += 32) {
        const double c = T[k / grid][k % grid];
        out[k] = c;
        out32[k] = __double2float_rn(c);
    }
    const int nc = grid >> 3;
    for (int k = lane; k < 32 * nc; k += 32) cdfc[t0 * nc + k] = __double2float_rn(T[k / nc][8 * (k % nc) + 7]);
}

// Members are read from `p` (positions, ID; region in reg) and their new
// state is written to `q` at slot dst(i) = map ? map[src_orig[i]] : i (the
// asynchronous batch reads a snapshot and writes the current arrays).
__global__ void k_remap(PArr p, PArr q, const int *__restrict__ src_orig, const int *__restrict__ map, int n,
                        const int *__restrict__ reg, const float *__restrict__ pred, int cout,
                        const double *__restrict__ cdf, const float *__restrict__ cdf32,
                        const float *__restrict__ cdfc, const double *__restrict__ cent, double side, double d,
                        double inv_d, int grid, const unsigned long long *__restrict__ seedp, int sweeps, int r0,
                        int r1)
{
    // members of regions [r0, r1); the line sums hold those regions
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int r = reg[i];
    if (r < r0 || r >= r1) return;
    uint64_t seed = *seedp;
    // d = side / grid and inv_d = 1 / d come from the host (two FP64
    // divides per thread would cost more than the rest of the FP64 work)
    double lo[3] = {cent[3 * r] - 0.5 * side, cent[3 * r + 1] - 0.5 * side, cent[3 * r + 2] - 0.5 * side};
    double pp[3] = {p.x[i], p.y[i], p.z[i]};
    int c[3];
    for (int a = 0; a < 3; a++) {
        // floor of the rounded quotient (q / d): q inv_d is within ~1e-14 of
        // it, so its floor is the same unless it lies within 1e-9 of an
        // integer, where the divide decides
        const double q = __dsub_rn(pp[a], lo[a]);
        const double g = q * inv_d;
        double f = floor(g);
        if (g - f < 1e-9 || f + 1.0 - g < 1e-9) f = floor(__ddiv_rn(q, d));
        c[a] = f < 0.0 ? 0 : (f > (double)(grid - 1) ? grid - 1 : (int)f);
    }
    const size_t G = (size_t)grid;
    uint64_t id = (uint64_t)p.id[i];
    const uint64_t sid = sm64(seed + id);  // the particle's stream: draw k is sm64(sid + k)
    const bool coarse8 = (grid & 31) == 0 && grid <= 64;  // lines of 8 or fewer coarse sums, float4-aligned
    uint64_t k = 0;
    for (int s = 0; s < sweeps; s++) {
        for (int a = 0; a < 3; a++, k++) {
            // the line through the current voxel along axis a; pick the first
            // q whose running sum exceeds target = U * total (the first
            // crossing of a scan of the non-decreasing running sums).  The
            // comparisons run on FP32 images: t32 approximates target from
            // the top 32 bits of U's 53-bit integer m and the FP32 total
            // within a relative 2^-21 (m >= 2^45: truncation 2^-24, three
            // roundings 2^-24 each, FP64 rounding of target 2^-53; the total
            // kept in FP32's normal range), and the FP32 sums are within 2^-24
            // of the FP64 ones, so a sum outside t32 (1 -+ 2^-20) orders
            // against target as its image does; inside that band (and for
            // m < 2^45) the FP64 values decide.  With 8 | grid the search is
            // two scans of 8: the coarse sums (every 8th) pick the block, the
            // block's 8 sums the voxel -- two dependent 32-byte loads.
            size_t line = a == 0 ? (size_t)c[2] * G + c[1] : (a == 1 ? (size_t)c[2] * G + c[0] : (size_t)c[1] * G + c[0]);
            const size_t lid = ((size_t)(r - r0) * 3 + a) * G * G + line;
            const double *L = cdf + lid * G;
            const float *L32 = cdf32 + lid * G;
            const uint64_t m = sm64(sid + k) >> 11;
            double target = 0.0;
            bool have = false;
            float lo32 = 0.f, hi32 = 0.f;
            bool fast = false;
            // true when running sum q (FP32 image l32) exceeds target
            auto above = [&](float l32, int q) -> bool {
                if (fast && l32 > hi32) return true;
                if (fast && l32 < lo32) return false;
                if (!have) {
                    target = __dmul_rn((double)m * (1.0 / 9007199254740992.0), L[grid - 1]);
                    have = true;
                }
                return L[q] > target;
            };
            auto setup = [&](float tot32) {
                fast = m >= (1ull << 45) && tot32 >= 0x1p-90f && tot32 <= 0x1p100f;
                // float(M), M = m >> 21 < 2^32, rounded to nearest, on the FP32
                // pipes: its two 16-bit halves are exact as 2^23 + x - 2^23, and
                // one FMA joins them with a single rounding
                const unsigned M = (unsigned)(m >> 21);
                const float mh = __int_as_float(0x4B000000 | (int)(M >> 16)) - 8388608.f;
                const float ml = __int_as_float(0x4B000000 | (int)(M & 0xFFFFu)) - 8388608.f;
                const float t32 = __fmul_rn(__fmaf_rn(mh, 65536.f, ml), tot32 * 0x1p-32f);
                lo32 = __fmul_rn(t32, 1.f - 0x1p-20f);
                hi32 = __fmul_rn(t32, 1.f + 0x1p-20f);
            };
            int qa;
            if (coarse8) {
                const int nc = grid >> 3;
                const float4 *C4 = reinterpret_cast<const float4 *>(cdfc + lid * nc);
                const float4 v0 = C4[0];
                const float4 v1 = nc == 8 ? C4[1] : v0;
                const float cv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
                setup(nc == 8 ? v1.w : v0.w);
                int jb = nc;
#pragma unroll
                for (int j = 0; j < 8; j++)
                    if (j < nc && above(cv[j], 8 * j + 7)) { jb = j; break; }
                if (jb == nc) {
                    qa = grid;
                } else {
                    const float4 *F4 = reinterpret_cast<const float4 *>(L32 + 8 * jb);
                    const float4 f0 = F4[0], f1 = F4[1];
                    const float fv[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
                    qa = 8 * jb + 7;  // block jb's last sum is above target
#pragma unroll
                    for (int q = 0; q < 7; q++)
                        if (above(fv[q], 8 * jb + q)) { qa = 8 * jb + q; break; }
                }
            } else {
                setup(L32[grid - 1]);
                int qb = grid;
                qa = 0;
                while (qa < qb) {
                    int mid = (qa + qb) >> 1;
                    if (above(L32[mid], mid)) qb = mid;
                    else qa = mid + 1;
                }
            }
            c[a] = qa < grid ? qa : grid - 1;
        }
    }
    double np[3];
    for (int a = 0; a < 3; a++) {
        np[a] = lo[a] + (c[a] + uniform_draw(sid, (uint64_t)(3 * sweeps + a))) * d;
    }
    const int o = map ? map[src_orig[i]] : i;
    q.x[o] = np[0];
    q.y[o] = np[1];
    q.z[o] = np[2];
    const float *pv = pred + ((((size_t)r * grid + c[2]) * grid + c[1]) * grid + c[0]) * cout;
    // u = 10^(2 z1 + 2) / T_PER_U in FP32: 2 z1 is exact, exp10f is within
    // 2 ulp, and the product with 100 / T_PER_U adds one rounding
    q.u[o] = exp10f(2.f * pv[1]) * (float)(100.0 / SUR_T_PER_U);
    q.vx[o] = 20.f * pv[2];
    q.vy[o] = 20.f * pv[3];
    q.vz[o] = 20.f * pv[4];
}

// ---------------------------------------------------------------- host
int voxelise_buffers_for(gnb_ctx *c, int nreg, int grid)
{
    size_t nv = (size_t)nreg * grid * grid * grid;
    if (c->sur_pcap < c->cap) {
        c->sur_gen++;
        dfree(c, c->sreg); dfree(c, c->vpa); dfree(c, c->vpb); dfree(c, c->vpc); dfree(c, c->vbox);
        c->sreg = nullptr; c->vpa = nullptr; c->vpb = nullptr; c->vpc = nullptr; c->vbox = nullptr;
        GNB_TRY(dalloc(c, &c->sreg, (size_t)c->cap + 1));
        GNB_TRY(dalloc(c, &c->vpa, (size_t)c->cap + 1));
        GNB_TRY(dalloc(c, &c->vpb, (size_t)c->cap + 1));
        GNB_TRY(dalloc(c, &c->vpc, (size_t)c->cap + 1));
        GNB_TRY(dalloc(c, &c->vbox, (size_t)c->cap + 1));
        c->sur_pcap = c->cap;
    }
    if (c->sur_nv < nv || c->sur_nreg < nreg) {
        c->sur_gen++;
        dfree(c, c->vacc); dfree(c, c->vw); dfree(c, c->vcdf); dfree(c, c->vcdf32); dfree(c, c->vcdfc);
        dfree(c, c->cent_d);
        dfree(c, c->rcount);
        dfree(c, c->vout); dfree(c, c->rsx); dfree(c, c->rsi); dfree(c, c->centf);
        c->vacc = nullptr; c->vw = nullptr; c->vcdf = nullptr; c->vcdf32 = nullptr; c->vcdfc = nullptr;
        c->cent_d = nullptr;
        c->rcount = nullptr;
        c->vout = nullptr; c->rsx = nullptr; c->rsi = nullptr; c->centf = nullptr;
        GNB_TRY(dalloc(c, &c->vacc, nv * 8));
        GNB_TRY(dalloc(c, &c->vw, nv));
        GNB_TRY(dalloc(c, &c->vcdf, nv * 3));
        GNB_TRY(dalloc(c, &c->vcdf32, nv * 3));
        GNB_TRY(dalloc(c, &c->vcdfc, nv * 3 / 8 + 1));
        GNB_TRY(dalloc(c, &c->vout, nv * 5));
        GNB_TRY(dalloc(c, &c->cent_d, (size_t)nreg * 3));
        GNB_TRY(dalloc(c, &c->rsx, (size_t)nreg));
        GNB_TRY(dalloc(c, &c->rsi, (size_t)nreg));
        GNB_TRY(dalloc(c, &c->centf, (size_t)nreg * 3));
        GNB_TRY(dalloc(c, &c->rcount, (size_t)nreg));
        c->sur_nv = nv;
        c->sur_nreg = nreg;
    }
    if (!c->seed_d) GNB_TRY(dalloc(c, &c->seed_d, 1));
    return GNB_OK;
}

// Centres to the device, with the regions sorted by centre x (ties by
// index) for the membership search.
static int upload_centres(gnb_ctx *c, int nreg, const double *centers)
{
    c->rs_order.resize(nreg);
    for (int k = 0; k < nreg; k++) c->rs_order[k] = k;
    std::sort(c->rs_order.begin(), c->rs_order.end(), [&](int a, int b) {
        return centers[3 * a] < centers[3 * b] || (centers[3 * a] == centers[3 * b] && a < b);
    });
    c->rs_x.resize(nreg);
    c->rs_cf.resize(3 * nreg);
    for (int k = 0; k < nreg; k++) c->rs_x[k] = (float)centers[3 * c->rs_order[k]];
    for (int k = 0; k < 3 * nreg; k++) c->rs_cf[k] = (float)centers[k];
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(c->cent_d, centers, sizeof(double) * 3 * nreg, cudaMemcpyHostToDevice,
                                          c->s), "centres"));
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(c->rsx, c->rs_x.data(), sizeof(float) * nreg, cudaMemcpyHostToDevice, c->s),
                       "sorted centres"));
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(c->centf, c->rs_cf.data(), sizeof(float) * 3 * nreg, cudaMemcpyHostToDevice,
                                          c->s), "FP32 centres"));
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(c->rsi, c->rs_order.data(), sizeof(int) * nreg, cudaMemcpyHostToDevice,
                                          c->s), "centre order"));
    return GNB_OK;
}

// Region membership of every gas particle (all nreg regions).
static void assign_launch(gnb_ctx *c, int nreg, double side, cudaStream_t st)
{
    int n = (int)c->n;
    cudaMemsetAsync(c->rcount, 0, sizeof(int) * nreg, st);
    counted(k_region_assign)<<<(n + 255) / 256, 256, 0, st>>>(c->P[c->cur], n, c->cent_d, c->rsx, c->rsi, c->centf,
                                                              nreg, 0.5 * side, c->sreg, c->rcount);
}

// Accumulators of regions [r0, r1) (membership already assigned); their
// finalised channels go to `out` (FP32 [nreg][grid^3][5]) and/or `outb`
// (BF16 U-Net input), both indexed from region 0.
// The members are read from the view (a, n, reg, rho): the context's current
// particles, or the asynchronous batch's snapshot.
static int vox_regions_view(gnb_ctx *c, const PArr &a, int n, const int *reg, const float *rho, int r0, int r1,
                            double side, int grid, float *out, bf16 *outb, cudaStream_t st)
{
    const long long V = (long long)grid * grid * grid;
    size_t nv = (size_t)(r1 - r0) * V;
    // accumulators: accA [nv][4], then accB [(nv + 1) / 2][4] (see k_vox_scatter)
    float *accA = c->vacc, *accB = c->vacc + nv * 4;
    cudaMemsetAsync(c->vacc, 0, sizeof(float) * (nv * 4 + (nv + 1) / 2 * 4), st);
    counted(k_vox_stage)<<<(n + 255) / 256, 256, 0, st>>>(a, n, reg, r0, r1, rho, c->cent_d, side, grid, c->vpa,
                                                          c->vpb, c->vpc, c->vbox);
    counted(k_vox_scatter)<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, reg, r0, r1, c->vpa, c->vpb, c->vpc,
                                                                       c->vbox, side, grid, accA, accB);
    for (int q0 = r0; q0 < r1; q0 += 65535) {  // gridDim.y holds at most 65,535 regions
        const int q1 = std::min(r1, q0 + 65535);
        counted(k_vox_finalize)<<<dim3((unsigned)((V + 255) / 256), (unsigned)(q1 - q0)), 256, 0, st>>>(
            accA, accB, (size_t)(q0 - r0) * V, (int)V, out ? out + (size_t)q0 * V * 5 : nullptr,
            outb ? outb + (size_t)q0 * V * 16 : nullptr);
    }
    GNB_LAUNCH_CHECK(c, "voxelise");
    return GNB_OK;
}

static int vox_regions(gnb_ctx *c, int r0, int r1, double side, int grid, float *out, bf16 *outb, cudaStream_t st)
{
    return vox_regions_view(c, c->P[c->cur], (int)c->n, c->sreg, c->rho, r0, r1, side, grid, out, outb, st);
}

static int vox_launch(gnb_ctx *c, int nreg, double side, int grid, float *out, bf16 *outb)
{
    assign_launch(c, nreg, side, c->s);
    return vox_regions(c, 0, nreg, side, grid, out, outb, c->s);
}

// Remap of the members of regions [r0, r1) from the predictions `pred`
// (FP32 [nreg][grid^3][cout], indexed from region 0).
static int remap_regions_launch(gnb_ctx *c, int r0, int r1, double side, int grid, const float *pred, int cout,
                                int sweeps, cudaStream_t st)
{
    int n = (int)c->n;
    const long long V = (long long)grid * grid * grid;
    size_t nv = (size_t)(r1 - r0) * V;
    counted(k_remap_weights)<<<(unsigned)((nv + 255) / 256), 256, 0, st>>>(pred + (size_t)r0 * V * cout,
                                                                           (long long)nv, cout, c->vw);
    long long nl = (long long)(r1 - r0) * 3 * grid * grid;
    if (grid == 32 || grid == 64)
        counted(k_line_cdf_tiled)<<<(unsigned)((nl / 32 + LC_W - 1) / LC_W), 32 * LC_W, 0, st>>>(
            c->vw, r1 - r0, grid, c->vcdf, c->vcdf32, c->vcdfc);
    else
        counted(k_line_cdf)<<<(unsigned)((nl + 127) / 128), 128, 0, st>>>(c->vw, r1 - r0, grid, c->vcdf, c->vcdf32,
                                                                          c->vcdfc);
    counted(k_remap)<<<(n + 127) / 128, 128, 0, st>>>(c->P[c->cur], c->P[c->cur], nullptr, nullptr, n, c->sreg, pred,
                                                      cout, c->vcdf, c->vcdf32,
                                                      c->vcdfc, c->cent_d, side, side / grid, 1.0 / (side / grid), grid,
                                                      c->seed_d, sweeps, r0, r1);
    GNB_LAUNCH_CHECK(c, "remap");
    return GNB_OK;
}

static int remap_launch(gnb_ctx *c, int nreg, double side, int grid, const float *pred, int cout, int sweeps)
{
    return remap_regions_launch(c, 0, nreg, side, grid, pred, cout, sweeps, c->s);
}

int voxelise(gnb_ctx *c, int nreg, const double *centers, double side, int grid, float *out_dev)
{
    GNB_TRY(voxelise_buffers_for(c, nreg, grid));
    GNB_TRY(upload_centres(c, nreg, centers));
    phase_begin(c, GNB_T_VOXELISE);
    int rc = vox_launch(c, nreg, side, grid, out_dev ? out_dev : c->vout, nullptr);
    phase_end(c);
    return rc;
}

int remap_regions(gnb_ctx *c, int nreg, const double *centers, double side, int grid, const float *pred_dev,
                  uint64_t seed, int sweeps)
{
    GNB_TRY(voxelise_buffers_for(c, nreg, grid));
    GNB_TRY(upload_centres(c, nreg, centers));
    unsigned long long sd = seed;
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(c->seed_d, &sd, sizeof(sd), cudaMemcpyHostToDevice, c->s), "seed"));
    int n = (int)c->n;
    cudaMemsetAsync(c->rcount, 0, sizeof(int) * nreg, c->s);
    counted(k_region_assign)<<<(n + 255) / 256, 256, 0, c->s>>>(c->P[c->cur], n, c->cent_d, c->rsx, c->rsi, c->centf,
                                                                nreg, 0.5 * side, c->sreg, c->rcount);
    phase_begin(c, GNB_T_REMAP);
    GNB_TRY(remap_launch(c, nreg, side, grid, pred_dev, 5, sweeps));
    phase_end(c);
    return cuda_check(c, cudaStreamSynchronize(c->s), "remap sync");
}

// ------------------------------------------------------- asynchronous batch
// The pool nodes' role (Sec. 3.2 steps 2-4): the members of the regions are
// snapshotted when the batch is submitted; voxelise, U-Net and the remap's
// line sums run on a side stream while the global steps go on; when the
// batch is applied (e.g. 50 global steps = 0.1 Myr later) each member, found
// by its caller index, is replaced by a draw from the predicted grid that
// starts from the voxel of its snapshot position.

__global__ void k_sna_flag(int n, const int *__restrict__ reg, int *__restrict__ flag)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = reg[i] >= 0;
}

// member i -> snapshot slot pos[i] (exclusive scan of the flags: Morton
// order kept, which keeps the voxel reductions local)
__global__ void k_sna_snapshot(PArr p, int n, const int *__restrict__ reg, const float *__restrict__ rho,
                               const int *__restrict__ pos, PArr s, float *__restrict__ srho, int *__restrict__ sreg,
                               int *__restrict__ sorig)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int r = reg[i];
    if (r < 0) return;
    const int k = pos[i];
    s.x[k] = p.x[i]; s.y[k] = p.y[i]; s.z[k] = p.z[i]; s.h2[k] = p.h2[i];
    s.m[k] = p.m[i]; s.u[k] = p.u[i]; s.vx[k] = p.vx[i]; s.vy[k] = p.vy[i]; s.vz[k] = p.vz[i];
    s.id[k] = p.id[i];
    srho[k] = rho[i];
    sreg[k] = r;
    sorig[k] = p.orig[i];
}

// current slot of every caller index
__global__ void k_inverse(const int *__restrict__ orig, int n, int *__restrict__ inv)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) inv[orig[i]] = i;
}

static PArr sna_view(gnb_ctx *c)
{
    PArr s;
    s.x = c->sna_x; s.y = c->sna_y; s.z = c->sna_z; s.h2 = c->sna_h2; s.id = c->sna_id;
    s.m = c->sna_m; s.u = c->sna_u; s.vx = c->sna_vx; s.vy = c->sna_vy; s.vz = c->sna_vz;
    return s;
}

static int sna_buffers(gnb_ctx *c)
{
    if (!c->sna_st) GNB_TRY(cuda_check(c, cudaStreamCreateWithFlags(&c->sna_st, cudaStreamNonBlocking), "stream"));
    if (!c->sna_ev_snap)
        GNB_TRY(cuda_check(c, cudaEventCreateWithFlags(&c->sna_ev_snap, cudaEventDisableTiming), "event"));
    if (!c->sna_ev_done)
        GNB_TRY(cuda_check(c, cudaEventCreateWithFlags(&c->sna_ev_done, cudaEventDisableTiming), "event"));
    if (!c->sna_seed) GNB_TRY(dalloc(c, &c->sna_seed, 1));
    if (c->sna_cap >= c->cap) return GNB_OK;
    void *old[] = {c->sna_x, c->sna_y, c->sna_z, c->sna_h2, c->sna_m, c->sna_u, c->sna_vx, c->sna_vy, c->sna_vz,
                   c->sna_rho, c->sna_reg, c->sna_orig, c->sna_pos, c->sna_inv, c->sna_id};
    for (void *q : old) dfree(c, q);
    const size_t m = (size_t)c->cap + 1;
    GNB_TRY(dalloc(c, &c->sna_x, m)); GNB_TRY(dalloc(c, &c->sna_y, m)); GNB_TRY(dalloc(c, &c->sna_z, m));
    GNB_TRY(dalloc(c, &c->sna_h2, m)); GNB_TRY(dalloc(c, &c->sna_m, m)); GNB_TRY(dalloc(c, &c->sna_u, m));
    GNB_TRY(dalloc(c, &c->sna_vx, m)); GNB_TRY(dalloc(c, &c->sna_vy, m)); GNB_TRY(dalloc(c, &c->sna_vz, m));
    GNB_TRY(dalloc(c, &c->sna_rho, m)); GNB_TRY(dalloc(c, &c->sna_reg, m)); GNB_TRY(dalloc(c, &c->sna_orig, m));
    GNB_TRY(dalloc(c, &c->sna_pos, m)); GNB_TRY(dalloc(c, &c->sna_inv, m)); GNB_TRY(dalloc(c, &c->sna_id, m));
    c->sna_cap = c->cap;
    return GNB_OK;
}

int sn_async_submit(gnb_ctx *c, gnb_unet *net, int nreg, const double *centers, double side, uint64_t seed,
                    int sweeps)
{
    if (c->sna_pending) return fail(c, GNB_ESTATE, "an asynchronous surrogate batch is already pending");
    bf16 *xin = nullptr;
    float *yout = nullptr;
    int grid = 0, cout = 0;
    GNB_TRY(unet_prepare(net, nreg, &xin, &yout, &grid, &cout));
    if (cout != 5) return fail(c, GNB_EINVAL, "the surrogate network must predict 5 channels");
    if (grid > 256) return fail(c, GNB_EINVAL, "surrogate grids are limited to 256 voxels per axis");
    GNB_TRY(voxelise_buffers_for(c, nreg, grid));
    GNB_TRY(upload_centres(c, nreg, centers));
    GNB_TRY(sna_buffers(c));
    unsigned long long sd = seed;
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(c->sna_seed, &sd, sizeof(sd), cudaMemcpyHostToDevice, c->s), "seed"));
    const int n = (int)c->n;
    const int nb = (n + 255) / 256;
    // snapshot on the context's stream
    assign_launch(c, nreg, side, c->s);
    counted(k_sna_flag)<<<nb, 256, 0, c->s>>>(n, c->sreg, c->sna_inv);
    GNB_TRY(device_scan(c, c->sna_inv, c->sna_pos, c->n_d, n, nullptr));
    cudaMemsetAsync(c->sna_reg, 0xff, sizeof(int) * (size_t)n, c->s);  // -1: not a member
    counted(k_sna_snapshot)<<<nb, 256, 0, c->s>>>(c->P[c->cur], n, c->sreg, c->rho, c->sna_pos, sna_view(c),
                                                  c->sna_rho, c->sna_reg, c->sna_orig);
    GNB_LAUNCH_CHECK(c, "surrogate snapshot");
    GNB_TRY(cuda_check(c, cudaEventRecord(c->sna_ev_snap, c->s), "event"));
    // the rest on the side stream
    cudaStream_t st = c->sna_st;
    GNB_TRY(cuda_check(c, cudaStreamWaitEvent(st, c->sna_ev_snap, 0), "event wait"));
    GNB_TRY(vox_regions_view(c, sna_view(c), n, c->sna_reg, c->sna_rho, 0, nreg, side, grid, nullptr, xin, st));
    GNB_TRY(unet_run(net, nreg, st, nullptr, nullptr));
    const size_t nv = (size_t)nreg * grid * grid * grid;
    counted(k_remap_weights)<<<(unsigned)((nv + 255) / 256), 256, 0, st>>>(yout, (long long)nv, cout, c->vw);
    const long long nl = (long long)nreg * 3 * grid * grid;
    if (grid == 32 || grid == 64)
        counted(k_line_cdf_tiled)<<<(unsigned)((nl / 32 + LC_W - 1) / LC_W), 32 * LC_W, 0, st>>>(
            c->vw, nreg, grid, c->vcdf, c->vcdf32, c->vcdfc);
    else
        counted(k_line_cdf)<<<(unsigned)((nl + 127) / 128), 128, 0, st>>>(c->vw, nreg, grid, c->vcdf, c->vcdf32,
                                                                          c->vcdfc);
    GNB_LAUNCH_CHECK(c, "surrogate side stream");
    GNB_TRY(cuda_check(c, cudaEventRecord(c->sna_ev_done, st), "event"));
    c->sna_pending = true;
    c->sna_nreg = nreg; c->sna_grid = grid; c->sna_sweeps = sweeps; c->sna_side = side;
    c->sna_net = net; c->sna_yout = yout;
    return GNB_OK;
}

int sn_async_apply(gnb_ctx *c)
{
    if (!c->sna_pending) return fail(c, GNB_ESTATE, "no asynchronous surrogate batch is pending");
    GNB_TRY(cuda_check(c, cudaStreamWaitEvent(c->s, c->sna_ev_done, 0), "event wait"));
    c->sna_pending = false;
    const int n = (int)c->n;
    const double side = c->sna_side;
    const int grid = c->sna_grid;
    counted(k_inverse)<<<(n + 255) / 256, 256, 0, c->s>>>(c->P[c->cur].orig, n, c->sna_inv);
    counted(k_remap)<<<(n + 127) / 128, 128, 0, c->s>>>(sna_view(c), c->P[c->cur], c->sna_orig, c->sna_inv, n,
                                                        c->sna_reg, c->sna_yout, 5, c->vcdf, c->vcdf32, c->vcdfc,
                                                        c->cent_d, side, side / grid, 1.0 / (side / grid), grid,
                                                        c->sna_seed, c->sna_sweeps, 0, c->sna_nreg);
    GNB_LAUNCH_CHECK(c, "surrogate apply");
    return GNB_OK;
}

// voxelise -> U-Net -> remap for nreg regions; after the first call with a
// given shape the whole sequence is replayed as one CUDA graph.
// The pipelined batch's two extra streams and its events, made once.
static int sn_streams(gnb_ctx *c)
{
    // the U-Net stream gets the highest priority and the remap stream the
    // next, so that their blocks are placed first as SMs free up
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    for (int k = 0; k < 2; k++)
        if (!c->sn_st[k])
            GNB_TRY(cuda_check(c, cudaStreamCreateWithPriority(&c->sn_st[k], cudaStreamNonBlocking,
                                                               k == 0 ? hi : (hi < lo ? hi + 1 : hi)), "stream"));
    for (auto &row : c->sn_ev)
        for (auto &e : row)
            if (!e) GNB_TRY(cuda_check(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event"));
    return GNB_OK;
}

int sn_surrogate_batch(gnb_ctx *c, gnb_unet *net, int nreg, const double *centers, double side, uint64_t seed,
                       int sweeps, int use_graph)
{
    bf16 *xin = nullptr;
    float *yout = nullptr;
    int grid = 0, cout = 0;
    GNB_TRY(unet_prepare(net, nreg, &xin, &yout, &grid, &cout));
    if (cout != 5) return fail(c, GNB_EINVAL, "the surrogate network must predict 5 channels");
    if (grid > 256) return fail(c, GNB_EINVAL, "surrogate grids are limited to 256 voxels per axis");
    GNB_TRY(voxelise_buffers_for(c, nreg, grid));
    GNB_TRY(upload_centres(c, nreg, centers));
    unsigned long long sd = seed;
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(c->seed_d, &sd, sizeof(sd), cudaMemcpyHostToDevice, c->s), "seed"));
    const int nch = std::max(1, std::min(std::min(c->sn_chunks, nreg), (int)gnb_ctx::SN_MAXCH));
    bool same = c->sn_graph && c->sn_key[0] == nreg && c->sn_key[1] == grid && c->sn_key[2] == sweeps &&
                c->sn_key[3] == nch &&
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
        GNB_TRY(unet_run(net, nreg, c->s, nullptr, nullptr));
        phase_begin(c, GNB_T_REMAP);
        int rc = remap_launch(c, nreg, side, grid, yout, cout, sweeps);
        phase_end(c);
        return rc;
    };
    // Pipelined (nch > 1): the regions go through in nch chunks; chunk k is
    // voxelised on the context's stream, runs through the U-Net on a second
    // stream and is remapped on a third, so the stages of different chunks
    // may overlap.  (On GB300 they gain nothing: the voxel scatter's L2
    // reductions and the remap's dependent L2 loads contend, and each stage
    // alone fills the GPU; the default is one chunk.)  The chunks' members are disjoint particles, every buffer is
    // used by one stream only (accumulators: voxelise; activations: U-Net;
    // line sums: remap) apart from the network's input and output, which
    // are indexed by region, and events order each chunk's three stages.
    const long long V = (long long)grid * grid * grid;
    auto issue_pipelined = [&]() -> int {
        GNB_TRY(sn_streams(c));
        cudaStream_t sa = c->s, sb = c->sn_st[0], sc = c->sn_st[1];
        assign_launch(c, nreg, side, sa);
        for (int k = 0; k < nch; k++) {
            const int r0 = (int)((long long)k * nreg / nch), r1 = (int)((long long)(k + 1) * nreg / nch);
            GNB_TRY(vox_regions(c, r0, r1, side, grid, nullptr, xin, sa));
            GNB_TRY(cuda_check(c, cudaEventRecord(c->sn_ev[0][k], sa), "event"));
            GNB_TRY(cuda_check(c, cudaStreamWaitEvent(sb, c->sn_ev[0][k], 0), "event wait"));
            GNB_TRY(unet_run(net, r1 - r0, sb, xin + (size_t)r0 * V * 16, yout + (size_t)r0 * V * cout));
            GNB_TRY(cuda_check(c, cudaEventRecord(c->sn_ev[1][k], sb), "event"));
            GNB_TRY(cuda_check(c, cudaStreamWaitEvent(sc, c->sn_ev[1][k], 0), "event wait"));
            GNB_TRY(remap_regions_launch(c, r0, r1, side, grid, yout, cout, sweeps, sc));
        }
        // join: the context's stream continues after the last remap
        GNB_TRY(cuda_check(c, cudaEventRecord(c->sn_ev[2][0], sc), "event"));
        return cuda_check(c, cudaStreamWaitEvent(sa, c->sn_ev[2][0], 0), "event wait");
    };
    // with the phase timers on, the batch runs eagerly and in sequence (no
    // graph, one chunk) so that each stage's events are recorded
    if (c->timing || c->s == nullptr) return issue();
    if (!use_graph) return nch > 1 ? issue_pipelined() : issue();
    if (c->sn_graph) {
        cudaGraphExecDestroy(c->sn_graph);
        c->sn_graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    GNB_TRY(cuda_check(c, cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal), "begin capture"));
    int rc = nch > 1 ? issue_pipelined() : issue();
    cudaError_t e = cudaStreamEndCapture(c->s, &g);
    if (rc != GNB_OK) { if (g) cudaGraphDestroy(g); return rc; }
    GNB_TRY(cuda_check(c, e, "end capture"));
    e = cudaGraphInstantiate(&c->sn_graph, g, 0);
    cudaGraphDestroy(g);
    GNB_TRY(cuda_check(c, e, "graph instantiate"));
    c->sn_key[0] = nreg; c->sn_key[1] = grid; c->sn_key[2] = sweeps; c->sn_key[3] = nch;
    c->sn_net = net; c->sn_side = side; c->sn_n = c->n; c->sn_cur = c->cur; c->sn_gen = c->sur_gen;
    return cuda_check(c, cudaGraphLaunch(c->sn_graph, c->s), "surrogate graph launch");
}

}  // namespace gnb
