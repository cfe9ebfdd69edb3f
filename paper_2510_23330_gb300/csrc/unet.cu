// unet.cu -- the supernova surrogate's 3D U-Net: BF16 inference and training
// kernels with FP32 accumulation (Sec. 3.3 of Hirashima et al., SC'25: a
// U-Net of 3D convolutions predicting the gas 0.1 Myr after a supernova,
// trained with an MSE loss and Adam at batch size 1).
//
// Architecture (a reading; the paper gives no layer list): levels with
// widths base, 2 base, 4 base, 8 base; two 3^3 convolutions (zero "same"
// padding, ReLU) per level; 2^3 max-pool down; 2^3 stride-2 transposed
// convolution up; skip tensor concatenated before the up-sampled tensor; 1^3
// linear head.  Activations are BF16 and blocked by 8 channels:
// [batch][channel / 8][z][y][x][channel % 8], so that 8 channels of one
// voxel are one 16-byte piece and a run of x voxels of one channel group is
// contiguous (the tensor-core convolution loads its halo rows by TMA); the
// network input is padded to 16 channels.
//
// Every convolution-shaped product is one implicit GEMM (rows = output
// voxels, columns = output channels, K = taps x input channels) on the
// tensor cores: BF16 operands staged in shared memory by cp.async (double
// buffered), mma.sync m16n8k16 with FP32 accumulators, bias/ReLU/BF16
// conversion fused into the epilogue.  Weight gradients are a second implicit
// GEMM (rows = input channels, K = voxels) split over voxel chunks.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "conv_tc.cuh"
#include "../../include/galnb_testing.h"

typedef __nv_bfloat16 bf16;

namespace gnb {

enum { IG_CONV3 = 0, IG_CONV1 = 1, IG_UP2 = 2, IG_DOWN2 = 3 };

__device__ __constant__ signed char c_taps[27][3] = {
    {-1, -1, -1}, {-1, -1, 0}, {-1, -1, 1}, {-1, 0, -1}, {-1, 0, 0}, {-1, 0, 1}, {-1, 1, -1}, {-1, 1, 0}, {-1, 1, 1},
    {0, -1, -1},  {0, -1, 0},  {0, -1, 1},  {0, 0, -1},  {0, 0, 0},  {0, 0, 1},  {0, 1, -1},  {0, 1, 0},  {0, 1, 1},
    {1, -1, -1},  {1, -1, 0},  {1, -1, 1},  {1, 0, -1},  {1, 0, 0},  {1, 0, 1},  {1, 1, -1},  {1, 1, 0},  {1, 1, 1}};

struct IgArgs {
    int mode;
    const bf16 *in1, *in2;  // input channels [0, C1) from in1, [C1, C1 + C2) from in2
    int C1, C2;
    const bf16 *w;          // [taps][Npad][K], K = C1 + C2
    const float *bias;      // [N] or null
    int N, Npad;
    bf16 *out1, *out2;      // channels [0, O1) -> out1, [O1, N) -> out2
    int O1;
    float *outf;            // FP32 output with N channels (instead of out1/out2)
    int relu;
    int B, D, H, W;         // grid of the GEMM rows
};

// Offset of element (voxel v = b * Vs + s, channel c) of a C-channel blocked
// tensor whose grid has Vs voxels per batch entry.
__device__ __forceinline__ long long blk(long long v, int c, int C, long long Vs)
{
    long long b = v / Vs, s = v - b * Vs;
    return ((b * (C >> 3) + (c >> 3)) * Vs + s) * 8 + (c & 7);
}

__device__ __forceinline__ void cp_async16(void *smem, const void *g, int bytes)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(g), "r"(bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void mma_bf16(float *d, const unsigned *a, const unsigned *b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Source voxel of GEMM row r for tap t (or -1 when it lies in the zero padding).
__device__ __forceinline__ long long ig_src(const IgArgs &p, long long r, int t)
{
    long long x = r % p.W, q = r / p.W;
    long long y = q % p.H;
    q /= p.H;
    long long z = q % p.D, b = q / p.D;
    if (p.mode == IG_CONV3) {
        long long zz = z + c_taps[t][0], yy = y + c_taps[t][1], xx = x + c_taps[t][2];
        if (zz < 0 || zz >= p.D || yy < 0 || yy >= p.H || xx < 0 || xx >= p.W) return -1;
        return ((b * p.D + zz) * p.H + yy) * p.W + xx;
    }
    if (p.mode == IG_DOWN2) {  // gather from the grid twice as fine
        long long zz = 2 * z + ((t >> 2) & 1), yy = 2 * y + ((t >> 1) & 1), xx = 2 * x + (t & 1);
        return ((b * 2 * p.D + zz) * 2 * p.H + yy) * 2 * p.W + xx;
    }
    return r;  // IG_CONV1, IG_UP2: the row's own voxel
}

// Output voxel of GEMM row r (IG_UP2 scatters into the grid twice as fine).
__device__ __forceinline__ long long ig_dst(const IgArgs &p, long long r, int t)
{
    if (p.mode != IG_UP2) return r;
    long long x = r % p.W, q = r / p.W;
    long long y = q % p.H;
    q /= p.H;
    long long z = q % p.D, b = q / p.D;
    long long zz = 2 * z + ((t >> 2) & 1), yy = 2 * y + ((t >> 1) & 1), xx = 2 * x + (t & 1);
    return ((b * 2 * p.D + zz) * 2 * p.H + yy) * 2 * p.W + xx;
}

#define IG_M 64
// NB = number of 8-column blocks per CTA (N tile = 8 NB)
template <int NB>
__global__ void __launch_bounds__(128) k_igemm(IgArgs p)
{
    constexpr int NT = 8 * NB;
    __shared__ __align__(16) bf16 sA[2][IG_M][16];
    __shared__ __align__(16) bf16 sB[2][NT][16];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gid = lane >> 2, tig = lane & 3;
    const long long M = (long long)p.B * p.D * p.H * p.W;
    const long long row0 = (long long)blockIdx.x * IG_M;
    const int n0 = blockIdx.y * NT;
    const int K = p.C1 + p.C2;
    const int ntap = p.mode == IG_CONV3 ? 27 : (p.mode == IG_DOWN2 ? 8 : 1);
    const int tapz = p.mode == IG_UP2 ? (int)blockIdx.z : 0;
    const int kch = K / 16;
    const int nsteps = ntap * kch;
    const long long Vrow = (long long)p.D * p.H * p.W;
    const long long VsA = p.mode == IG_DOWN2 ? 8 * Vrow : Vrow;  // voxels per batch entry of the source grid
    const long long VsO = p.mode == IG_UP2 ? 8 * Vrow : Vrow;    // ... and of the output grid
    float acc[NB][4];
#pragma unroll
    for (int j = 0; j < NB; j++) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;

    auto stage = [&](int s, int buf) {
        int t = s / kch, c0 = (s % kch) * 16;
        int wt = p.mode == IG_UP2 ? tapz : t;
        {   // A: 64 rows x 16 channels, one 16-byte piece per thread
            int r = tid >> 1, half = tid & 1;
            long long gr = row0 + r;
            long long v = gr < M ? ig_src(p, gr, t) : -1;
            int c = c0 + 8 * half;
            const bf16 *src = p.in1;
            int bytes = 0;
            if (v >= 0) {
                src = c < p.C1 ? p.in1 + blk(v, c, p.C1, VsA) : p.in2 + blk(v, c - p.C1, p.C2, VsA);
                bytes = 16;
            }
            cp_async16(&sA[buf][r][8 * half], src, bytes);
        }
        for (int q = tid; q < NT * 2; q += 128) {  // B: NT rows x 16 k
            int n = q >> 1, half = q & 1;
            bool in = (n0 + n) < p.Npad;
            const bf16 *src = in ? p.w + ((long long)wt * p.Npad + n0 + n) * K + c0 + 8 * half : p.w;
            cp_async16(&sB[buf][n][8 * half], src, in ? 16 : 0);
        }
        cp_async_commit();
    };

    stage(0, 0);
    for (int s = 0; s < nsteps; s++) {
        const int buf = s & 1;
        if (s + 1 < nsteps) {
            stage(s + 1, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        unsigned a[4];
        const int ra = 16 * warp + gid;
        a[0] = *reinterpret_cast<const unsigned *>(&sA[buf][ra][2 * tig]);
        a[1] = *reinterpret_cast<const unsigned *>(&sA[buf][ra + 8][2 * tig]);
        a[2] = *reinterpret_cast<const unsigned *>(&sA[buf][ra][2 * tig + 8]);
        a[3] = *reinterpret_cast<const unsigned *>(&sA[buf][ra + 8][2 * tig + 8]);
#pragma unroll
        for (int j = 0; j < NB; j++) {
            unsigned b[2];
            b[0] = *reinterpret_cast<const unsigned *>(&sB[buf][8 * j + gid][2 * tig]);
            b[1] = *reinterpret_cast<const unsigned *>(&sB[buf][8 * j + gid][2 * tig + 8]);
            mma_bf16(acc[j], a, b);
        }
        __syncthreads();
    }
    // epilogue: bias, ReLU, BF16 (or FP32) store
#pragma unroll
    for (int h = 0; h < 2; h++) {
        long long gr = row0 + 16 * warp + gid + 8 * h;
        if (gr >= M) continue;
        long long ov = ig_dst(p, gr, tapz);
#pragma unroll
        for (int j = 0; j < NB; j++) {
            int col = n0 + 8 * j + 2 * tig;
            float v0 = acc[j][2 * h], v1 = acc[j][2 * h + 1];
            if (p.bias) {
                if (col < p.N) v0 += p.bias[col];
                if (col + 1 < p.N) v1 += p.bias[col + 1];
            }
            if (p.relu) { v0 = fmaxf(v0, 0.f); v1 = fmaxf(v1, 0.f); }
            if (p.outf) {
                if (col < p.N) p.outf[ov * p.N + col] = v0;
                if (col + 1 < p.N) p.outf[ov * p.N + col + 1] = v1;
            } else if (col + 1 < p.N || (col < p.N && (p.N & 1) == 0)) {
                __nv_bfloat162 pr = __floats2bfloat162_rn(v0, v1);
                if (col < p.O1) *reinterpret_cast<__nv_bfloat162 *>(p.out1 + blk(ov, col, p.O1, VsO)) = pr;
                else *reinterpret_cast<__nv_bfloat162 *>(p.out2 + blk(ov, col - p.O1, p.N - p.O1, VsO)) = pr;
            }
        }
    }
}

// Weight gradient dW[tap][ci][co] += sum_v X(v, tap)[ci] * G(v, tap)[co] over a
// chunk of GEMM rows v (split-K with FP32 atomics).  X is the forward input
// (concatenated from two tensors), G the output gradient.
struct WgArgs {
    int mode;
    const bf16 *x1, *x2;
    int C1, C2;
    const bf16 *g;
    int Cg;          // channels stored in g (>= N, multiple of 8)
    int N;           // output channels that exist in dW
    int Cw;          // input channels that exist in dW (<= C1 + C2; the padded network input has more)
    float *dw;       // [taps][Cw][N]
    int B, D, H, W;  // grid of the rows (coarse grid for IG_UP2)
    long long chunk; // rows per CTA
};

template <int NB>
__global__ void __launch_bounds__(128) k_wgrad(WgArgs p)
{
    constexpr int NT = 8 * NB;
    __shared__ __align__(16) bf16 sX[64][16 + 2];
    __shared__ __align__(16) bf16 sG[NT][16 + 2];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gid = lane >> 2, tig = lane & 3;
    const long long M = (long long)p.B * p.D * p.H * p.W;
    const int t = blockIdx.z;
    const int ci0 = blockIdx.y * 64;
    const int Cin = p.C1 + p.C2;
    const long long r0 = (long long)blockIdx.x * p.chunk, r1 = min(M, r0 + p.chunk);
    IgArgs q;
    q.mode = p.mode; q.B = p.B; q.D = p.D; q.H = p.H; q.W = p.W;
    const long long VsX = (long long)p.D * p.H * p.W;                    // X lives on the row grid
    const long long VsG = p.mode == IG_UP2 ? 8 * VsX : VsX;              // G on the fine grid for IG_UP2
    float acc[NB][4];
#pragma unroll
    for (int j = 0; j < NB; j++) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    for (long long rb = r0; rb < r1; rb += 16) {
        // X tile: 16 rows x 64 input channels, stored transposed [ci][row]
        for (int e = tid; e < 16 * 8; e += 128) {
            int rr = e >> 3, c8 = (e & 7) * 8;
            long long r = rb + rr;
            long long v = -1;
            if (r < r1) v = p.mode == IG_UP2 ? r : ig_src(q, r, t);
            int c = ci0 + c8;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (v >= 0 && c < Cin)
                val = c < p.C1 ? *reinterpret_cast<const uint4 *>(p.x1 + blk(v, c, p.C1, VsX))
                               : *reinterpret_cast<const uint4 *>(p.x2 + blk(v, c - p.C1, p.C2, VsX));
            const bf16 *pv = reinterpret_cast<const bf16 *>(&val);
#pragma unroll
            for (int k = 0; k < 8; k++) sX[c8 + k][rr] = pv[k];
        }
        // G tile: 16 rows x NT output channels, stored transposed [co][row]
        for (int e = tid; e < 16 * NB; e += 128) {
            int rr = e / NB, c8 = (e % NB) * 8;
            long long r = rb + rr;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (r < r1) {
                long long v = p.mode == IG_UP2 ? ig_dst(q, r, t) : r;
                if (c8 < p.Cg) val = *reinterpret_cast<const uint4 *>(p.g + blk(v, c8, p.Cg, VsG));
            }
            const bf16 *pv = reinterpret_cast<const bf16 *>(&val);
#pragma unroll
            for (int k = 0; k < 8; k++) sG[c8 + k][rr] = pv[k];
        }
        __syncthreads();
        unsigned a[4];
        const int ra = 16 * warp + gid;
        a[0] = *reinterpret_cast<const unsigned *>(&sX[ra][2 * tig]);
        a[1] = *reinterpret_cast<const unsigned *>(&sX[ra + 8][2 * tig]);
        a[2] = *reinterpret_cast<const unsigned *>(&sX[ra][2 * tig + 8]);
        a[3] = *reinterpret_cast<const unsigned *>(&sX[ra + 8][2 * tig + 8]);
#pragma unroll
        for (int j = 0; j < NB; j++) {
            unsigned b[2];
            b[0] = *reinterpret_cast<const unsigned *>(&sG[8 * j + gid][2 * tig]);
            b[1] = *reinterpret_cast<const unsigned *>(&sG[8 * j + gid][2 * tig + 8]);
            mma_bf16(acc[j], a, b);
        }
        __syncthreads();
    }
#pragma unroll
    for (int h = 0; h < 2; h++) {
        int ci = ci0 + 16 * warp + gid + 8 * h;
        if (ci >= p.Cw) continue;
#pragma unroll
        for (int j = 0; j < NB; j++) {
            int co = 8 * j + 2 * tig;
            float *d = p.dw + ((long long)t * p.Cw + ci) * p.N;
            if (co < p.N) atomicAdd(d + co, acc[j][2 * h]);
            if (co + 1 < p.N) atomicAdd(d + co + 1, acc[j][2 * h + 1]);
        }
    }
}

// ----------------------------------------------------------------- elementwise
// FP32 [V][cin] -> blocked BF16 with 16 channels (zeros beyond cin); Vs
// voxels per batch entry.
__global__ void k_pack_input(const float *__restrict__ x, int cin, long long V, long long Vs, bf16 *__restrict__ out)
{
    // one voxel per thread: its cin values, two 16-byte channel groups out
    long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    float f[16];
#pragma unroll
    for (int c = 0; c < 16; c++) f[c] = c < cin ? x[v * cin + c] : 0.f;
    const long long b = v / Vs, sv = v - b * Vs;
#pragma unroll
    for (int g = 0; g < 2; g++) {
        uint4 o;
        unsigned *ou = reinterpret_cast<unsigned *>(&o);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            __nv_bfloat162 h = __floats2bfloat162_rn(f[8 * g + 2 * q], f[8 * g + 2 * q + 1]);
            ou[q] = *reinterpret_cast<unsigned *>(&h);
        }
        *reinterpret_cast<uint4 *>(out + ((b * 2 + g) * Vs + sv) * 8) = o;
    }
}

// 1x1x1 head: FP32 out[v][n] = bias[n] + sum_k in(v)[k] w[n][k] for n < cout
// (<= 8) and k < C (<= 32, a multiple of 8); w is the packed BF16 [Npad][Kpad]
// forward weight.  One voxel per thread; a block's outputs are staged in
// shared memory and leave as contiguous 16-byte stores.
constexpr int HEAD_T = 256;
__global__ void __launch_bounds__(HEAD_T) k_head(const bf16 *__restrict__ in, int C, const bf16 *__restrict__ w,
                                                 int Kpad, const float *__restrict__ bias, int cout, long long V,
                                                 long long Vs, float *__restrict__ out)
{
    __shared__ float sw[8][32], sbias[8];
    __shared__ __align__(16) float so[HEAD_T * 8];
    for (int i = threadIdx.x; i < 8 * 32; i += blockDim.x) {
        const int n = i >> 5, k = i & 31;
        sw[n][k] = n < cout && k < C ? __bfloat162float(w[n * Kpad + k]) : 0.f;
    }
    if (threadIdx.x < 8) sbias[threadIdx.x] = threadIdx.x < cout && bias ? bias[threadIdx.x] : 0.f;
    __syncthreads();
    const long long v0 = (long long)blockIdx.x * HEAD_T;
    const long long v = v0 + threadIdx.x;
    if (v < V) {
        const long long b = v / Vs, sv = v - b * Vs;
        float acc[8];
#pragma unroll
        for (int n = 0; n < 8; n++) acc[n] = sbias[n];
#pragma unroll
        for (int g = 0; g < 4; g++) {
            if (g >= (C >> 3)) break;
            const uint4 u = *reinterpret_cast<const uint4 *>(in + ((b * (C >> 3) + g) * Vs + sv) * 8);
            const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const float2 f = __bfloat1622float2(h[q]);
#pragma unroll
                for (int n = 0; n < 8; n++) acc[n] += f.x * sw[n][8 * g + 2 * q] + f.y * sw[n][8 * g + 2 * q + 1];
            }
        }
#pragma unroll
        for (int n = 0; n < 8; n++)
            if (n < cout) so[threadIdx.x * cout + n] = acc[n];
    }
    __syncthreads();
    const long long nv = V - v0 < HEAD_T ? V - v0 : HEAD_T;
    const long long nf = nv * cout;  // floats of this block, contiguous from out + v0 cout
    float *dst = out + v0 * cout;
    if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
        for (long long i = threadIdx.x; i < nf / 4; i += HEAD_T)
            reinterpret_cast<float4 *>(dst)[i] = reinterpret_cast<const float4 *>(so)[i];
        for (long long i = (nf / 4) * 4 + threadIdx.x; i < nf; i += HEAD_T) dst[i] = so[i];
    } else {
        for (long long i = threadIdx.x; i < nf; i += HEAD_T) dst[i] = so[i];
    }
}

__global__ void k_maxpool(const bf16 *__restrict__ in, bf16 *__restrict__ out, unsigned char *__restrict__ idx, int B,
                          int D, int H, int W, int C)
{
    // output grid (B, D, H, W); input grid twice as fine; q runs over the
    // blocked output's (b, channel group, voxel): 8 channels per thread, the
    // 2x2x2 inputs as 16-byte loads; the first maximum of the 8 taps wins
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long Vs = (long long)D * H * W;
    if (q >= (long long)B * (C >> 3) * Vs) return;
    long long s = q % Vs, bg = q / Vs;  // bg = b * C / 8 + channel group
    long long x = s % W, r = s / W, y = r % H, z = r / H;
    const bf16 *src = in + bg * 8 * Vs * 8;
    float best[8];
    unsigned bi[8];
#pragma unroll
    for (int t = 0; t < 8; t++) {
        long long zz = 2 * z + ((t >> 2) & 1), yy = 2 * y + ((t >> 1) & 1), xx = 2 * x + (t & 1);
        const uint4 u = *reinterpret_cast<const uint4 *>(src + ((zz * 2 * H + yy) * 2 * W + xx) * 8);
        const bf16 *h = reinterpret_cast<const bf16 *>(&u);
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const float f = __bfloat162float(h[j]);
            if (t == 0 || f > best[j]) { best[j] = f; bi[j] = (unsigned)t; }
        }
    }
    uint4 o;
    bf16 *ob = reinterpret_cast<bf16 *>(&o);
    unsigned lo = 0, hi = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        ob[j] = __float2bfloat16_rn(best[j]);
        if (j < 4) lo |= bi[j] << (8 * j);
        else hi |= bi[j] << (8 * (j - 4));
    }
    *reinterpret_cast<uint4 *>(out + q * 8) = o;
    *reinterpret_cast<uint2 *>(idx + q * 8) = make_uint2(lo, hi);
}

// dIn (fine grid) = routed pool gradient + skip gradient
__global__ void k_maxpool_bwd(const bf16 *__restrict__ dout, const unsigned char *__restrict__ idx,
                              const bf16 *__restrict__ dskip, bf16 *__restrict__ din, int B, int D, int H, int W, int C)
{
    // fine grid (B, 2D, 2H, 2W); e runs over the blocked fine tensor
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tot = (long long)B * 8 * D * H * W * C;
    if (e >= tot) return;
    const long long Vc = (long long)D * H * W, Vf = 8 * Vc;
    int j = (int)(e & 7);
    long long q = e >> 3;
    long long s = q % Vf, bg = q / Vf;
    long long x = s % (2 * W), r = s / (2 * W), y = r % (2 * H), z = r / (2 * H);
    int t = (int)(((z & 1) << 2) | ((y & 1) << 1) | (x & 1));
    long long cv = (bg * Vc + ((z >> 1) * H + (y >> 1)) * W + (x >> 1)) * 8 + j;
    float g = idx[cv] == t ? __bfloat162float(dout[cv]) : 0.f;
    if (dskip) g += __bfloat162float(dskip[e]);
    din[e] = __float2bfloat16_rn(g);
}

// Blocked BF16 [B][C/8][V][8] -> FP32 [B][V][keep] (the first `keep` channels).
__global__ void k_unblock(const bf16 *__restrict__ in, int B, int C, long long V, int keep, float *__restrict__ out)
{
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)B * V * keep) return;
    int c = (int)(e % keep);
    long long bv = e / keep, b = bv / V, v = bv - b * V;
    out[e] = __bfloat162float(in[((b * (C >> 3) + (c >> 3)) * V + v) * 8 + (c & 7)]);
}

__global__ void k_relu_mask(const bf16 *__restrict__ dy, const bf16 *__restrict__ y, bf16 *__restrict__ dz, long long n)
{
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) dz[e] = __bfloat162float(y[e]) > 0.f ? dy[e] : __float2bfloat16_rn(0.f);
}

// MSE over (voxels, cout): loss partial sums in FP64 and dy = 2 (y - t) / count
// as BF16 with 16 channels (zeros beyond cout).
__global__ void k_mse(const float *__restrict__ y, const float *__restrict__ tgt, long long V, long long Vs, int cout,
                      bf16 *__restrict__ dy, double *__restrict__ loss)
{
    __shared__ double sh[32];
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (e < V * 16) {
        long long v = e >> 4;
        int c = (int)(e & 15);
        float g = 0.f;
        if (c < cout) {
            float d = y[v * cout + c] - tgt[v * cout + c];
            l = (double)d * d;
            g = 2.f * d / (float)(V * cout);
        }
        dy[blk(v, c, 16, Vs)] = __float2bfloat16_rn(g);
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) s += sh[q];
        atomicAdd(loss, s);
    }
}

// column sums of a blocked BF16 tensor with Cs channels (V voxels, Vs per
// batch entry) into db[0..N)
__global__ void k_colsum(const bf16 *__restrict__ g, long long V, long long Vs, int Cs, int N, float *__restrict__ db)
{
    int c = threadIdx.x % Cs;
    int lanes = blockDim.x / Cs;
    int sub = threadIdx.x / Cs;
    if (sub >= lanes) return;
    float s = 0.f;
    for (long long v = (long long)blockIdx.x * lanes + sub; v < V; v += (long long)gridDim.x * lanes)
        s += __bfloat162float(g[blk(v, c, Cs, Vs)]);
    if (c < N) atomicAdd(&db[c], s);
}

// Adam (Kingma and Ba): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
// p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).  The constants
// 1 - b1, 1 - b2 and the bias corrections 1 / (1 - b^t) come from the host in
// FP64, rounded once: formed in FP32, 1 - 0.999f and 1 - 0.999^t lose five
// significant digits to cancellation.
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, long long n, float lr, float b1, float ob1, float b2, float ob2,
                       float eps, float ic1, float ic2)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    float mi = __fmaf_rn(b1, m[i], ob1 * gi);
    float vi = __fmaf_rn(b2, v[i], ob2 * (gi * gi));
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * ic1) / (sqrtf(vi * ic2) + eps);
}

// master [taps][cin][cout] FP32 -> forward BF16 [taps][Npad][Kpad] (transposed, zero padded)
__global__ void k_pack_w_fwd(const float *__restrict__ w, int taps, int cin, int cout, int Npad, int Kpad,
                             bf16 *__restrict__ out)
{
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tot = (long long)taps * Npad * Kpad;
    if (e >= tot) return;
    int k = (int)(e % Kpad);
    long long q = e / Kpad;
    int n = (int)(q % Npad);
    int t = (int)(q / Npad);
    out[e] = __float2bfloat16_rn(k < cin && n < cout ? w[((long long)t * cin + k) * cout + n] : 0.f);
}

// master -> input-gradient BF16 [taps][Npad = cin_pad][Kpad = cout_pad]; taps of a 3^3
// convolution are mirrored (tap t -> 26 - t)
__global__ void k_pack_w_dgrad(const float *__restrict__ w, int taps, int mirror, int cin, int cout, int Npad,
                               int Kpad, bf16 *__restrict__ out)
{
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tot = (long long)taps * Npad * Kpad;
    if (e >= tot) return;
    int k = (int)(e % Kpad);
    long long q = e / Kpad;
    int n = (int)(q % Npad);
    int t = (int)(q / Npad);
    int ts = mirror ? taps - 1 - t : t;
    out[e] = __float2bfloat16_rn(k < cout && n < cin ? w[((long long)ts * cin + n) * cout + k] : 0.f);
}

}  // namespace gnb

// =================================================================== host
using namespace gnb;

namespace {

enum { L_CONV3 = 0, L_UP2 = 1, L_CONV1 = 2 };

struct ULayer {
    mutable int plan_f = -1;    // tile plan of the tensor-core forward convolution (-1: the rule's choice)
    int kind, cin, cout, taps;
    long long woff, boff;       // offsets in the flat parameter array
    int Npad, Kpad, Nd, Kd;     // padded forward / input-gradient GEMM shapes
    bf16 *wf = nullptr, *wd = nullptr;
    bf16 *wtc = nullptr, *wdtc = nullptr;  // tensor-core layouts of wf / wd (3^3 and up-sampling layers)
};

int round_up(int a, int b) { return (a + b - 1) / b * b; }

}  // namespace

struct gnb_unet {
    int cin, cout, base, levels, grid;
    cudaStream_t s;
    std::vector<ULayer> L;
    long long nparam = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    int adam_t = 0;
    // activations for batch capacity bcap
    int bcap = 0;
    std::vector<bf16 *> act;     // per stored tensor
    std::vector<unsigned char *> pidx;
    bf16 *xin = nullptr;
    float *yout = nullptr, *tgt = nullptr;
    bf16 *dyb = nullptr;
    std::vector<bf16 *> tmp;     // backward scratch
    double *loss_d = nullptr;
    int *err_d = nullptr;        // device error word of the tcgen05 convolutions
    int conv_impl = GNB_CONV_AUTO;
    unsigned tx_extra = 0;       // wait-timeout test only
    bool launch_failed = false;
    bool tuning = false;         // forward passes time every tile plan of each 3^3 layer (gnb_unet_autotune)
    int tuned_layers = 0;
    std::string err;
};

namespace {

void unet_free_acts(gnb_unet *u)
{
    for (auto *a : u->act) if (a) cudaFree(a);
    for (auto *a : u->pidx) if (a) cudaFree(a);
    for (auto *a : u->tmp) if (a) cudaFree(a);
    u->act.clear(); u->pidx.clear(); u->tmp.clear();
    if (u->xin) cudaFree(u->xin);
    if (u->yout) cudaFree(u->yout);
    if (u->tgt) cudaFree(u->tgt);
    if (u->dyb) cudaFree(u->dyb);
    u->xin = nullptr; u->yout = nullptr; u->tgt = nullptr; u->dyb = nullptr;
    u->bcap = 0;
}

// Tensor slots (index into act): per level l: 4 l + {0: enc a, 1: enc b (skip), 2: pool out}
// decoder level l: base 4 * levels + 3 l + {0: up, 1: dec a, 2: dec b}
int S_ENCA(int l) { return 4 * l; }
int S_ENCB(int l) { return 4 * l + 1; }
int S_POOL(int l) { return 4 * l + 2; }
int S_UP(const gnb_unet *u, int l) { return 4 * u->levels + 3 * l; }
int S_DECA(const gnb_unet *u, int l) { return 4 * u->levels + 3 * l + 1; }
int S_DECB(const gnb_unet *u, int l) { return 4 * u->levels + 3 * l + 2; }

int width(const gnb_unet *u, int l) { return u->base << l; }
long long vox(const gnb_unet *u, int l, int B) { long long g = u->grid >> l; return (long long)B * g * g * g; }

int unet_alloc_acts(gnb_unet *u, int B)
{
    if (u->bcap >= B) return GNB_OK;
    unet_free_acts(u);
    int nslot = 4 * u->levels + 3 * u->levels;
    u->act.assign(nslot, nullptr);
    u->pidx.assign(u->levels, nullptr);
    auto al = [&](void **p, size_t bytes) { return cudaMalloc(p, bytes) == cudaSuccess; };
    bool ok = true;
    for (int l = 0; l < u->levels; l++) {
        size_t n = (size_t)vox(u, l, B) * width(u, l);
        ok &= al((void **)&u->act[S_ENCA(l)], n * 2) && al((void **)&u->act[S_ENCB(l)], n * 2);
        if (l + 1 < u->levels) {
            size_t np = (size_t)vox(u, l + 1, B) * width(u, l);
            ok &= al((void **)&u->act[S_POOL(l)], np * 2) && al((void **)&u->pidx[l], np);
        }
        if (l + 1 < u->levels) {
            ok &= al((void **)&u->act[S_UP(u, l)], n * 2) && al((void **)&u->act[S_DECA(u, l)], n * 2) &&
                  al((void **)&u->act[S_DECB(u, l)], n * 2);
        }
    }
    size_t v0 = (size_t)vox(u, 0, B);
    ok &= al((void **)&u->xin, v0 * 16 * 2) && al((void **)&u->yout, v0 * u->cout * 4) &&
          al((void **)&u->tgt, v0 * u->cout * 4) && al((void **)&u->dyb, v0 * 16 * 2);
    // backward scratch: 4 buffers of the largest level-0 tensor with 2 * base channels
    u->tmp.assign(4, nullptr);
    for (int k = 0; k < 4; k++) ok &= al((void **)&u->tmp[k], v0 * (size_t)(2 * u->base) * 2 + 256);
    if (!ok) {
        cudaGetLastError();
        unet_free_acts(u);
        return GNB_ENOMEM;
    }
    u->bcap = B;
    return GNB_OK;
}

template <int NB>
void launch_ig_nb(const IgArgs &a, int ntiles_n, int gz, cudaStream_t s)
{
    long long M = (long long)a.B * a.D * a.H * a.W;
    dim3 grid((unsigned)((M + IG_M - 1) / IG_M), ntiles_n, gz);
    counted(k_igemm<NB>)<<<grid, 128, 0, s>>>(a);
}

void launch_ig(const IgArgs &a, cudaStream_t s)
{
    int gz = a.mode == IG_UP2 ? 8 : 1;
    int Np = a.Npad;
    if (Np <= 8) launch_ig_nb<1>(a, 1, gz, s);
    else if (Np <= 16) launch_ig_nb<2>(a, 1, gz, s);
    else if (Np <= 32) launch_ig_nb<4>(a, 1, gz, s);
    else if (Np <= 64) launch_ig_nb<8>(a, 1, gz, s);
    else launch_ig_nb<16>(a, (Np + 127) / 128, gz, s);
}

template <int NB>
void launch_wg_nb(const WgArgs &a, int taps, cudaStream_t s)
{
    long long M = (long long)a.B * a.D * a.H * a.W;
    int cin = a.C1 + a.C2;
    dim3 grid((unsigned)((M + a.chunk - 1) / a.chunk), (cin + 63) / 64, taps);
    counted(k_wgrad<NB>)<<<grid, 128, 0, s>>>(a);
}

void launch_wg(WgArgs a, int taps, cudaStream_t s)
{
    long long M = (long long)a.B * a.D * a.H * a.W;
    long long want = M / 96 + 1;  // about 96 chunks per tap
    a.chunk = ((want + 15) / 16) * 16;
    if (a.chunk < 256) a.chunk = 256;
    int Np = round_up(a.N, 8);
    if (Np <= 8) launch_wg_nb<1>(a, taps, s);
    else if (Np <= 16) launch_wg_nb<2>(a, taps, s);
    else if (Np <= 32) launch_wg_nb<4>(a, taps, s);
    else if (Np <= 64) launch_wg_nb<8>(a, taps, s);
    else launch_wg_nb<16>(a, taps, s);
}

IgArgs ig_base(int mode, int B, int D, int H, int W)
{
    IgArgs a;
    memset(&a, 0, sizeof(a));
    a.mode = mode; a.B = B; a.D = D; a.H = H; a.W = W;
    return a;
}

int unet_pack(gnb_unet *u)
{
    for (auto &l : u->L) {
        long long nf = (long long)l.taps * l.Npad * l.Kpad;
        counted(k_pack_w_fwd)<<<(unsigned)((nf + 255) / 256), 256, 0, u->s>>>(u->p + l.woff, l.taps, l.cin, l.cout,
                                                                            l.Npad, l.Kpad, l.wf);
        long long nd = (long long)l.taps * l.Nd * l.Kd;
        counted(k_pack_w_dgrad)<<<(unsigned)((nd + 255) / 256), 256, 0, u->s>>>(
            u->p + l.woff, l.taps, l.kind == L_CONV3 ? 1 : 0, l.cin, l.cout, l.Nd, l.Kd, l.wd);
        // up-sampling: the 8 taps' output channels are the rows of one matrix
        if (l.wtc && l.kind == L_UP2 && pack_w_tc(l.wf, 1, 8 * l.Npad, l.Kpad, l.wtc, u->s) != 0) return GNB_ECUDA;
        if (l.wtc && l.kind == L_CONV3 && pack_w_tc(l.wf, l.taps, l.Npad, l.Kpad, l.wtc, u->s) != 0) return GNB_ECUDA;
        if (l.wdtc && pack_w_tc(l.wd, l.taps, l.Nd, l.Kd, l.wdtc, u->s) != 0) return GNB_ECUDA;
    }
    return cudaGetLastError() == cudaSuccess ? GNB_OK : GNB_ECUDA;
}

// layer index helpers (order of the flat parameter array)
int LI_ENCA(int l) { return 2 * l; }
int LI_ENCB(int l) { return 2 * l + 1; }
int LI_UP(const gnb_unet *u, int l) { return 2 * u->levels + 3 * (u->levels - 2 - l); }
int LI_DECA(const gnb_unet *u, int l) { return LI_UP(u, l) + 1; }
int LI_DECB(const gnb_unet *u, int l) { return LI_UP(u, l) + 2; }
int LI_HEAD(const gnb_unet *u) { return 2 * u->levels + 3 * (u->levels - 1); }

// The tcgen05 path for a 3^3 convolution: 1 launched, 0 not applicable, -1 error.
int conv3_try_tc(gnb_unet *u, const bf16 *wtc, int N, int B, int D, const bf16 *in1, int C1, const bf16 *in2, int C2,
                 const float *bias, bf16 *out1, int O1, bf16 *out2, int relu, int plan = -1)
{
    if (!wtc || u->conv_impl == GNB_CONV_MMA_SYNC) return 0;
    TcConv c;
    c.plan = plan;
    c.in1 = in1; c.in2 = in2 ? in2 : in1; c.C1 = C1; c.C2 = C2;
    c.w = wtc; c.bias = bias; c.N = N;
    c.out1 = out1; c.out2 = out2 ? out2 : out1; c.O1 = O1; c.relu = relu;
    c.B = B; c.D = D; c.H = D; c.W = D;
    c.tx_extra = u->tx_extra;
    u->tx_extra = 0;  // the wait-timeout test affects the first tensor-core launch only
    return conv3_tc(c, u->err_d, u->s);
}

// Tile autotuner of one tensor-core 3^3 layer: every supported plan (tile
// depth, halo buffers, resident or streamed weights) runs on the layer's real
// tensors, twice untimed and three times timed with CUDA events on the
// network's stream, and the fastest is kept for the layer's forward passes.
void tune_conv3(gnb_unet *u, const ULayer &ly, int B, int D, const bf16 *in1, int C1, const bf16 *in2, int C2,
                bf16 *out, int relu)
{
    TcPlan plans[TC_MAX_PLANS];
    const int np = conv3_tc_plans(ly.Npad, C1 + C2, D, plans, TC_MAX_PLANS);
    if (np < 2) return;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return; }
    float best = 3.0e38f;
    int bi = -1;
    for (int k = 0; k < np; k++) {
        bool ok = true;
        for (int rep = 0; rep < 5 && ok; rep++) {
            if (rep == 2) cudaEventRecord(e0, u->s);
            ok = conv3_try_tc(u, ly.wtc, ly.Npad, B, D, in1, C1, in2, C2, u->p + ly.boff, out, ly.cout, nullptr, relu,
                              k) == 1;
        }
        cudaEventRecord(e1, u->s);
        float ms = 0.f;
        if (ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
            ms < best) {
            best = ms;
            bi = k;
        }
    }
    cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (bi >= 0) ly.plan_f = bi;
    u->tuned_layers++;
}

void conv_fwd(gnb_unet *u, const ULayer &ly, int mode, int B, int D, const bf16 *in1, int C1, const bf16 *in2, int C2,
              bf16 *out, float *outf, int relu)
{
    if (mode == IG_CONV3 && !outf) {
        if (u->tuning && ly.wtc && u->conv_impl != GNB_CONV_MMA_SYNC) tune_conv3(u, ly, B, D, in1, C1, in2, C2, out, relu);
        int rc = conv3_try_tc(u, ly.wtc, ly.Npad, B, D, in1, C1, in2, C2, u->p + ly.boff, out, ly.cout, nullptr,
                              relu, ly.plan_f);
        if (rc != 0) { if (rc < 0) u->launch_failed = true; return; }
    }
    if (mode == IG_UP2 && !outf && !in2 && !relu && ly.wtc && C1 == ly.Kpad && ly.cout == ly.Npad &&
        u->conv_impl != GNB_CONV_MMA_SYNC) {
        int rc = up2_tc(in1, ly.wtc, u->p + ly.boff, out, B, D, C1, ly.Npad, u->err_d, u->s);
        if (rc != 0) { if (rc < 0) u->launch_failed = true; return; }
    }
    if (mode == IG_CONV1 && outf && !in2 && ly.Npad <= 8 && C1 % 8 == 0 && C1 <= 32 && ly.Kpad <= 32) {
        const long long V = (long long)B * D * D * D;
        counted(k_head)<<<(unsigned)((V + HEAD_T - 1) / HEAD_T), HEAD_T, 0, u->s>>>(in1, C1, ly.wf, ly.Kpad, u->p + ly.boff, ly.cout,
                                                                      V, (long long)D * D * D, outf);
        return;
    }
    IgArgs a = ig_base(mode, B, D, D, D);
    a.in1 = in1; a.in2 = in2 ? in2 : in1; a.C1 = C1; a.C2 = C2;
    a.w = ly.wf; a.bias = u->p + ly.boff; a.N = ly.cout; a.Npad = ly.Npad;
    a.out1 = out; a.out2 = out; a.O1 = ly.cout; a.outf = outf; a.relu = relu;
    launch_ig(a, u->s);
}

// input gradient of a layer: dx (split in two when the input was a concatenation)
void conv_dgrad(gnb_unet *u, const ULayer &ly, int mode, int B, int D, const bf16 *dz, int Cz, bf16 *dx1, int O1,
                bf16 *dx2)
{
    if (mode == IG_CONV3 && Cz == ly.Kd) {
        int rc = conv3_try_tc(u, ly.wdtc, ly.Nd, B, D, dz, Cz, nullptr, 0, nullptr, dx1, O1, dx2, 0);
        if (rc != 0) { if (rc < 0) u->launch_failed = true; return; }
    }
    IgArgs a = ig_base(mode, B, D, D, D);
    a.in1 = dz; a.in2 = dz; a.C1 = Cz; a.C2 = 0;
    a.w = ly.wd; a.bias = nullptr; a.N = ly.cin; a.Npad = ly.Nd;
    a.out1 = dx1; a.out2 = dx2 ? dx2 : dx1; a.O1 = O1; a.outf = nullptr; a.relu = 0;
    launch_ig(a, u->s);
}

void conv_wgrad(gnb_unet *u, const ULayer &ly, int mode, int B, int D, const bf16 *x1, int C1, const bf16 *x2, int C2,
                const bf16 *g, int Cg)
{
    WgArgs a;
    memset(&a, 0, sizeof(a));
    a.mode = mode; a.x1 = x1; a.x2 = x2 ? x2 : x1; a.C1 = C1; a.C2 = C2; a.g = g; a.Cg = Cg; a.N = ly.cout;
    a.Cw = ly.cin;
    a.dw = u->g + ly.woff; a.B = B; a.D = D; a.H = D; a.W = D;
    // 3^3 layers on the tensor cores where the shape allows (tcgen05 GEMM
    // over (tap, channel) rows); the mma.sync GEMM otherwise
    int tc = 0;
    if (mode == IG_CONV3 && u->conv_impl == GNB_CONV_AUTO) {
        tc = wgrad3_tc(x1, C1, x2, x2 ? C2 : 0, g, Cg, ly.cout, ly.cin, a.dw, B, D, u->err_d, u->s);
        if (tc < 0) u->launch_failed = true;
    }
    if (tc == 0) launch_wg(a, ly.taps, u->s);
    // bias gradient: column sums of the output gradient
    long long Vs = mode == IG_UP2 ? 8LL * D * D * D : (long long)D * D * D;
    long long V = (long long)B * Vs;
    int threads = 256 / Cg * Cg;
    if (threads < Cg) threads = Cg;
    counted(k_colsum)<<<120, threads, 0, u->s>>>(g, V, Vs, Cg, ly.cout, u->g + ly.boff);
}

// Forward pass of B regions from the blocked BF16 input xin to the FP32
// output yout (defaults: the network's own buffers).
int unet_forward(gnb_unet *u, int B, const bf16 *xin = nullptr, float *yout = nullptr)
{
    int G = u->grid;
    const bf16 *h = xin ? xin : u->xin;
    int ch = 16;
    for (int l = 0; l < u->levels; l++) {
        int D = G >> l, w = width(u, l);
        conv_fwd(u, u->L[LI_ENCA(l)], IG_CONV3, B, D, h, ch, nullptr, 0, u->act[S_ENCA(l)], nullptr, 1);
        conv_fwd(u, u->L[LI_ENCB(l)], IG_CONV3, B, D, u->act[S_ENCA(l)], w, nullptr, 0, u->act[S_ENCB(l)], nullptr, 1);
        if (l + 1 < u->levels) {
            long long n = vox(u, l + 1, B) * w;
            counted(k_maxpool)<<<(unsigned)((n / 8 + 255) / 256), 256, 0, u->s>>>(u->act[S_ENCB(l)], u->act[S_POOL(l)],
                                                                                 u->pidx[l], B, D / 2, D / 2, D / 2, w);
            h = u->act[S_POOL(l)];
        } else {
            h = u->act[S_ENCB(l)];
        }
        ch = w;
    }
    for (int l = u->levels - 2; l >= 0; l--) {
        int D = G >> l, w = width(u, l);
        // up-sampling GEMM rows live on the coarse grid
        conv_fwd(u, u->L[LI_UP(u, l)], IG_UP2, B, D / 2, h, 2 * w, nullptr, 0, u->act[S_UP(u, l)], nullptr, 0);
        conv_fwd(u, u->L[LI_DECA(u, l)], IG_CONV3, B, D, u->act[S_ENCB(l)], w, u->act[S_UP(u, l)], w,
                 u->act[S_DECA(u, l)], nullptr, 1);
        conv_fwd(u, u->L[LI_DECB(u, l)], IG_CONV3, B, D, u->act[S_DECA(u, l)], w, nullptr, 0, u->act[S_DECB(u, l)],
                 nullptr, 1);
        h = u->act[S_DECB(u, l)];
    }
    conv_fwd(u, u->L[LI_HEAD(u)], IG_CONV1, B, G, h, u->base, nullptr, 0, nullptr, yout ? yout : u->yout, 0);
    return cudaGetLastError() == cudaSuccess && !u->launch_failed ? GNB_OK : GNB_ECUDA;
}

// Backward through the network for dy in u->dyb (16 channels); gradients
// accumulate into u->g (zeroed by the caller).
int unet_backward(gnb_unet *u, int B)
{
    int G = u->grid, b0 = u->base;
    cudaStream_t s = u->s;
    bf16 *T0 = u->tmp[0], *T1 = u->tmp[1], *T2 = u->tmp[2], *T3 = u->tmp[3];
    auto relu_mask = [&](const bf16 *dy, const bf16 *y, bf16 *dz, long long n) {
        counted(k_relu_mask)<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dy, y, dz, n);
    };
    // head
    const ULayer &hd = u->L[LI_HEAD(u)];
    const bf16 *top = u->act[S_DECB(u, 0)];
    conv_wgrad(u, hd, IG_CONV1, B, G, top, b0, nullptr, 0, u->dyb, 16);
    conv_dgrad(u, hd, IG_CONV1, B, G, u->dyb, 16, T0, b0, nullptr);  // T0: d(dec0b.out)
    // decoder levels 0 .. levels-2; skip gradients stay in the ENC slots' spare: use T-buffers per level
    // dskip[l] is stored in place of the decoder's "up" activation gradient area: allocate per level below
    std::vector<bf16 *> dskip(u->levels, nullptr);
    bf16 *dcur = T0;  // gradient of the current decoder output
    for (int l = 0; l + 1 < u->levels; l++) {
        int D = G >> l, w = width(u, l);
        long long n = vox(u, l, B) * w;
        // the level-l tensors are at most as large as level 0 with 2 * base channels
        relu_mask(dcur, u->act[S_DECB(u, l)], T1, n);
        conv_wgrad(u, u->L[LI_DECB(u, l)], IG_CONV3, B, D, u->act[S_DECA(u, l)], w, nullptr, 0, T1, w);
        conv_dgrad(u, u->L[LI_DECB(u, l)], IG_CONV3, B, D, T1, w, T2, w, nullptr);
        relu_mask(T2, u->act[S_DECA(u, l)], T1, n);
        conv_wgrad(u, u->L[LI_DECA(u, l)], IG_CONV3, B, D, u->act[S_ENCB(l)], w, u->act[S_UP(u, l)], w, T1, w);
        // dskip -> the level's dec-a slot (its forward value is no longer needed), dup -> T2
        dskip[l] = u->act[S_DECA(u, l)];
        conv_dgrad(u, u->L[LI_DECA(u, l)], IG_CONV3, B, D, T1, w, dskip[l], w, T2);
        // up-conv: weight gradient (rows on the coarse grid), input gradient by gather
        int Dc = D / 2, wc = 2 * w;
        conv_wgrad(u, u->L[LI_UP(u, l)], IG_UP2, B, Dc, l + 2 < u->levels ? u->act[S_DECB(u, l + 1)]
                                                                          : u->act[S_ENCB(u->levels - 1)],
                   wc, nullptr, 0, T2, w);
        conv_dgrad(u, u->L[LI_UP(u, l)], IG_DOWN2, B, Dc, T2, w, T3, wc, nullptr);
        std::swap(T0, T3);
        dcur = T0;  // gradient of the level-(l+1) decoder output (or the bottleneck)
    }
    // encoder, bottleneck first
    for (int l = u->levels - 1; l >= 0; l--) {
        int D = G >> l, w = width(u, l);
        long long n = vox(u, l, B) * w;
        if (l + 1 < u->levels) {
            // dcur is the gradient of pool(l) output; route it and add the skip gradient
            counted(k_maxpool_bwd)<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dcur, u->pidx[l], dskip[l], T3, B,
                                                                             D / 2, D / 2, D / 2, w);
            std::swap(T0, T3);
            dcur = T0;
        }
        relu_mask(dcur, u->act[S_ENCB(l)], T1, n);
        conv_wgrad(u, u->L[LI_ENCB(l)], IG_CONV3, B, D, u->act[S_ENCA(l)], w, nullptr, 0, T1, w);
        conv_dgrad(u, u->L[LI_ENCB(l)], IG_CONV3, B, D, T1, w, T2, w, nullptr);
        relu_mask(T2, u->act[S_ENCA(l)], T1, n);
        const bf16 *xin = l == 0 ? u->xin : u->act[S_POOL(l - 1)];
        int cin = l == 0 ? 16 : width(u, l - 1);
        conv_wgrad(u, u->L[LI_ENCA(l)], IG_CONV3, B, D, xin, cin, nullptr, 0, T1, w);
        if (l > 0) {
            conv_dgrad(u, u->L[LI_ENCA(l)], IG_CONV3, B, D, T1, w, T3, cin, nullptr);
            std::swap(T0, T3);
            dcur = T0;
        }
    }
    return cudaGetLastError() == cudaSuccess && !u->launch_failed ? GNB_OK : GNB_ECUDA;
}

// Synchronise and collect errors: launch failures, CUDA errors and the
// tcgen05 convolutions' device error word (a bounded wait that ran out).
int unet_check(gnb_unet *u, int rc)
{
    u->launch_failed = false;
    if (cudaStreamSynchronize(u->s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return GNB_ECUDA;
    int e = 0;
    if (u->err_d) {
        if (cudaMemcpy(&e, u->err_d, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return GNB_ECUDA;
        if (e != 0) {
            cudaMemsetAsync(u->err_d, 0, sizeof(int), u->s);
            cudaStreamSynchronize(u->s);
            return GNB_ETIMEOUT;
        }
    }
    return rc;
}

}  // namespace

namespace gnb {
// Hooks for the batched surrogate step: make room for `batch` regions and
// expose the blocked BF16 input [batch][2][grid^3][8] and the FP32 output
// [batch][grid^3][cout]; unet_run launches the forward pass of `batch`
// regions on `stream` without synchronising (so it can be captured in a CUDA
// graph), from xin to yout (null: those buffers' starts).
int unet_prepare(gnb_unet *u, int batch, bf16 **xin, float **yout, int *grid, int *cout)
{
    int rc = unet_alloc_acts(u, batch);
    if (rc != GNB_OK) return rc;
    *xin = u->xin;
    *yout = u->yout;
    *grid = u->grid;
    *cout = u->cout;
    return GNB_OK;
}

int unet_poll_error(gnb_unet *u)
{
    int e = 0;
    if (!u || !u->err_d || cudaMemcpy(&e, u->err_d, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return GNB_OK;
    if (e == 0) return GNB_OK;
    cudaMemsetAsync(u->err_d, 0, sizeof(int), u->s);
    return GNB_ETIMEOUT;
}

int unet_run(gnb_unet *u, int batch, cudaStream_t stream, const bf16 *xin, float *yout)
{
    cudaStream_t keep = u->s;
    u->s = stream;
    int rc = unet_forward(u, batch, xin, yout);
    u->s = keep;
    return rc;
}
}  // namespace gnb

extern "C" {

int gnb_unet_create(gnb_unet **out, int cin, int cout, int base, int levels, int grid, void *stream)
{
    if (!out) return GNB_EINVAL;
    *out = nullptr;
    if (cin < 1 || cin > 16 || cout < 1 || cout > 8 || base < 8 || base > 32 || (base % 8) || levels < 2 ||
        levels > 5 || grid < 8 || (grid % (1 << (levels - 1))) || ((grid >> (levels - 1)) < 2))
        return GNB_EINVAL;
    gnb_unet *u = new (std::nothrow) gnb_unet();
    if (!u) return GNB_ENOMEM;
    u->cin = cin; u->cout = cout; u->base = base; u->levels = levels; u->grid = grid;
    u->s = (cudaStream_t)stream;
    // layers in the order of the flat parameter array
    auto add = [&](int kind, int ci, int co) {
        ULayer l;
        l.kind = kind; l.cin = ci; l.cout = co;
        l.taps = kind == L_CONV3 ? 27 : (kind == L_UP2 ? 8 : 1);
        l.woff = u->nparam;
        u->nparam += (long long)l.taps * ci * co;
        l.boff = u->nparam;
        u->nparam += co;
        l.Kpad = round_up(ci, 16);
        l.Npad = round_up(co, 8);
        l.Nd = round_up(ci, 8);
        l.Kd = round_up(co, 16);
        u->L.push_back(l);
    };
    int c = 16;  // the network input is padded to 16 channels
    for (int l = 0; l < levels; l++) {
        add(L_CONV3, l == 0 ? cin : c, base << l);
        add(L_CONV3, base << l, base << l);
        c = base << l;
    }
    for (int l = levels - 2; l >= 0; l--) {
        add(L_UP2, base << (l + 1), base << l);
        add(L_CONV3, 2 * (base << l), base << l);
        add(L_CONV3, base << l, base << l);
    }
    add(L_CONV1, base, cout);
    // the first layer's input has 16 (padded) channels in the GEMM
    u->L[0].Kpad = 16;
    u->L[0].Nd = 16;
    bool ok = cudaMalloc((void **)&u->p, u->nparam * 4) == cudaSuccess &&
              cudaMalloc((void **)&u->g, u->nparam * 4) == cudaSuccess &&
              cudaMalloc((void **)&u->m, u->nparam * 4) == cudaSuccess &&
              cudaMalloc((void **)&u->v, u->nparam * 4) == cudaSuccess &&
              cudaMalloc((void **)&u->loss_d, 16) == cudaSuccess &&
              cudaMalloc((void **)&u->err_d, sizeof(int)) == cudaSuccess;
    for (auto &l : u->L) {
        ok = ok && cudaMalloc((void **)&l.wf, (size_t)l.taps * l.Npad * l.Kpad * 2) == cudaSuccess &&
             cudaMalloc((void **)&l.wd, (size_t)l.taps * l.Nd * l.Kd * 2) == cudaSuccess;
        TcPlan pl;
        if (ok && l.kind == L_CONV3 && conv3_tc_plan(l.Npad, l.Kpad, grid, &pl))
            ok = cudaMalloc((void **)&l.wtc, (size_t)l.taps * l.Npad * l.Kpad * 2) == cudaSuccess;
        if (ok && l.kind == L_UP2 && l.cin == l.Kpad && up2_tc_ok(l.Npad, l.Kpad, 128))
            ok = cudaMalloc((void **)&l.wtc, (size_t)l.taps * l.Npad * l.Kpad * 2) == cudaSuccess;
        if (ok && l.kind == L_CONV3 && conv3_tc_plan(l.Nd, l.Kd, grid, &pl))
            ok = cudaMalloc((void **)&l.wdtc, (size_t)l.taps * l.Nd * l.Kd * 2) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        gnb_unet_destroy(u);
        return GNB_ENOMEM;
    }
    cudaMemsetAsync(u->p, 0, u->nparam * 4, u->s);
    cudaMemsetAsync(u->g, 0, u->nparam * 4, u->s);
    cudaMemsetAsync(u->m, 0, u->nparam * 4, u->s);
    cudaMemsetAsync(u->v, 0, u->nparam * 4, u->s);
    cudaMemsetAsync(u->err_d, 0, sizeof(int), u->s);
    *out = u;
    return unet_check(u, unet_pack(u));
}

void gnb_unet_destroy(gnb_unet *u)
{
    if (!u) return;
    cudaStreamSynchronize(u->s);
    unet_free_acts(u);
    for (auto &l : u->L) {
        if (l.wf) cudaFree(l.wf);
        if (l.wd) cudaFree(l.wd);
        if (l.wtc) cudaFree(l.wtc);
        if (l.wdtc) cudaFree(l.wdtc);
    }
    float *a[] = {u->p, u->g, u->m, u->v};
    for (float *q : a) if (q) cudaFree(q);
    if (u->loss_d) cudaFree(u->loss_d);
    if (u->err_d) cudaFree(u->err_d);
    delete u;
}

int64_t gnb_unet_num_params(const gnb_unet *u) { return u ? u->nparam : -1; }

int gnb_unet_test_wait_timeout(gnb_unet *u)
{
    if (!u || u->conv_impl == GNB_CONV_MMA_SYNC) return GNB_EINVAL;
    int rc = unet_alloc_acts(u, 1);
    if (rc != GNB_OK) return rc;
    cudaMemsetAsync(u->xin, 0, (size_t)vox(u, 0, 1) * 16 * 2, u->s);
    u->tx_extra = 16;
    rc = unet_forward(u, 1);
    u->tx_extra = 0;
    return unet_check(u, rc);
}

int gnb_unet_set_conv_impl(gnb_unet *u, int impl)
{
    if (!u || (impl != GNB_CONV_AUTO && impl != GNB_CONV_MMA_SYNC)) return GNB_EINVAL;
    u->conv_impl = impl;
    return GNB_OK;
}

int gnb_unet_get_params(gnb_unet *u, float *dst, int on_device)
{
    if (!u || !dst) return GNB_EINVAL;
    cudaMemcpyAsync(dst, u->p, u->nparam * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, u->s);
    return unet_check(u, GNB_OK);
}

int gnb_unet_get_grads(gnb_unet *u, float *dst, int on_device)
{
    if (!u || !dst) return GNB_EINVAL;
    cudaMemcpyAsync(dst, u->g, u->nparam * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, u->s);
    return unet_check(u, GNB_OK);
}

int gnb_unet_get_activation(gnb_unet *u, int slot, int batch, float *dst, int on_device)
{
    if (!u || !dst || batch < 1 || batch > u->bcap || slot < 0) return GNB_EINVAL;
    // slot order: the input, then per level enc a, enc b (and the pooled
    // tensor below the coarsest level), then per decoder level (coarse to
    // fine) up, dec a, dec b
    const bf16 *src = nullptr;
    int C = 0, keep = 0, lev = 0;
    int k = slot;
    if (k == 0) {
        src = u->xin; C = 16; keep = u->cin; lev = 0;
    } else {
        k -= 1;
        for (int l = 0; l < u->levels && !src; l++) {
            const int w = width(u, l);
            const int nl = l + 1 < u->levels ? 3 : 2;
            if (k < nl) {
                src = u->act[k == 0 ? S_ENCA(l) : k == 1 ? S_ENCB(l) : S_POOL(l)];
                C = keep = w;
                lev = k == 2 ? l + 1 : l;
            }
            k -= nl;
        }
        for (int l = u->levels - 2; l >= 0 && !src; l--) {
            if (k < 3) {
                src = u->act[k == 0 ? S_UP(u, l) : k == 1 ? S_DECA(u, l) : S_DECB(u, l)];
                C = keep = width(u, l);
                lev = l;
            }
            k -= 3;
        }
    }
    if (!src) return GNB_EINVAL;
    const long long V = vox(u, lev, 1);
    const long long n = (long long)batch * V * keep;
    float *out = dst, *tmp = nullptr;
    if (!on_device) {
        if (cudaMalloc((void **)&tmp, n * 4) != cudaSuccess) {
            cudaGetLastError();
            return GNB_ENOMEM;
        }
        out = tmp;
    }
    counted(k_unblock)<<<(unsigned)((n + 255) / 256), 256, 0, u->s>>>(src, batch, C, V, keep, out);
    if (!on_device) cudaMemcpyAsync(dst, tmp, n * 4, cudaMemcpyDeviceToHost, u->s);
    int rc = unet_check(u, GNB_OK);
    if (tmp) cudaFree(tmp);
    return rc;
}

int gnb_unet_autotune(gnb_unet *u, int batch, double out_ms[2])
{
    if (!u || batch < 1) return GNB_EINVAL;
    int rc = unet_alloc_acts(u, batch);
    if (rc != GNB_OK) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return GNB_ECUDA;
    }
    auto timed = [&](double *ms) -> int {
        for (int w = 0; w < 2; w++) {
            int r = unet_forward(u, batch);
            if (r != GNB_OK) return r;
        }
        cudaEventRecord(e0, u->s);
        for (int w = 0; w < 3; w++) {
            int r = unet_forward(u, batch);
            if (r != GNB_OK) return r;
        }
        cudaEventRecord(e1, u->s);
        float f = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&f, e0, e1) != cudaSuccess) return GNB_ECUDA;
        *ms = f / 3.0;
        return GNB_OK;
    };
    for (auto &ly : u->L) ly.plan_f = -1;
    double before = 0.0, after = 0.0;
    rc = timed(&before);
    if (rc == GNB_OK) {
        u->tuning = true;
        u->tuned_layers = 0;
        rc = unet_forward(u, batch);
        u->tuning = false;
    }
    if (rc == GNB_OK) rc = timed(&after);
    if (rc == GNB_OK && after > before)  // the timings of single layers did not add up: keep the rule
        for (auto &ly : u->L) ly.plan_f = -1;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (out_ms) {
        out_ms[0] = before;
        out_ms[1] = after;
    }
    return unet_check(u, rc);
}

int gnb_unet_get_output(gnb_unet *u, int batch, float *dst, int on_device)
{
    if (!u || !dst || batch < 1 || batch > u->bcap || !u->yout) return GNB_EINVAL;
    size_t bytes = (size_t)vox(u, 0, batch) * u->cout * 4;
    cudaMemcpyAsync(dst, u->yout, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, u->s);
    return unet_check(u, GNB_OK);
}

int gnb_unet_set_params(gnb_unet *u, const float *src, int on_device)
{
    if (!u || !src) return GNB_EINVAL;
    cudaMemcpyAsync(u->p, src, u->nparam * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, u->s);
    cudaMemsetAsync(u->m, 0, u->nparam * 4, u->s);
    cudaMemsetAsync(u->v, 0, u->nparam * 4, u->s);
    u->adam_t = 0;
    return unet_check(u, unet_pack(u));
}

// Checkpoint of a network: a 64-byte header ("GNBUNET1", uint32 version 1,
// int32 cin, cout, base, levels, grid, int64 parameter count, int64 Adam
// steps taken, zero padding), then the FP32 master parameters and Adam's
// first and second moments, each [parameter count], in the order of
// gnb_unet_get_params.
namespace {
struct UnetCkHeader {
    char magic[8];
    uint32_t version;
    int32_t cin, cout, base, levels, grid;
    int64_t nparam, adam_t;
    unsigned char pad[64 - 8 - 4 - 20 - 16];
};
static_assert(sizeof(UnetCkHeader) == 64, "network checkpoint header is 64 bytes");
constexpr char UNET_MAGIC[8] = {'G', 'N', 'B', 'U', 'N', 'E', 'T', '1'};
}  // namespace

int gnb_unet_save(gnb_unet *u, const char *path)
{
    if (!u || !path) return GNB_EINVAL;
    std::vector<float> host((size_t)u->nparam * 3);
    for (int k = 0; k < 3; k++) {
        const float *src = k == 0 ? u->p : (k == 1 ? u->m : u->v);
        cudaMemcpyAsync(host.data() + (size_t)k * u->nparam, src, u->nparam * 4, cudaMemcpyDeviceToHost, u->s);
    }
    const int rc = unet_check(u, GNB_OK);
    if (rc != GNB_OK) return rc;
    UnetCkHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, UNET_MAGIC, 8);
    h.version = 1;
    h.cin = u->cin; h.cout = u->cout; h.base = u->base; h.levels = u->levels; h.grid = u->grid;
    h.nparam = u->nparam;
    h.adam_t = u->adam_t;
    FILE *f = fopen(path, "wb");
    if (!f) return GNB_EINVAL;
    const bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(host.data(), 4, host.size(), f) == host.size();
    const bool closed = fclose(f) == 0;
    return ok && closed ? GNB_OK : GNB_EINVAL;
}

int gnb_unet_load(gnb_unet *u, const char *path)
{
    if (!u || !path) return GNB_EINVAL;
    FILE *f = fopen(path, "rb");
    if (!f) return GNB_EINVAL;
    UnetCkHeader h;
    std::vector<float> host;
    int rc = GNB_OK;
    if (fread(&h, sizeof(h), 1, f) != 1 || memcmp(h.magic, UNET_MAGIC, 8) != 0 || h.version != 1) {
        rc = GNB_EINVAL;
    } else if (h.cin != u->cin || h.cout != u->cout || h.base != u->base || h.levels != u->levels ||
               h.grid != u->grid || h.nparam != u->nparam || h.adam_t < 0) {
        rc = GNB_EMISMATCH;
    } else {
        host.resize((size_t)u->nparam * 3);
        if (fread(host.data(), 4, host.size(), f) != host.size()) rc = GNB_EINVAL;
    }
    fclose(f);
    if (rc != GNB_OK) return rc;
    for (int k = 0; k < 3; k++) {
        float *dst = k == 0 ? u->p : (k == 1 ? u->m : u->v);
        cudaMemcpyAsync(dst, host.data() + (size_t)k * u->nparam, u->nparam * 4, cudaMemcpyHostToDevice, u->s);
    }
    u->adam_t = (int)h.adam_t;
    return unet_check(u, unet_pack(u));
}

int gnb_unet_forward(gnb_unet *u, int batch, const float *x, float *y, int on_device)
{
    if (!u || !x || !y || batch < 1) return GNB_EINVAL;
    int rc = unet_alloc_acts(u, batch);
    if (rc != GNB_OK) return rc;
    long long V = vox(u, 0, batch);
    const float *xd = x;
    float *tmpx = nullptr;
    if (!on_device) {
        if (cudaMalloc((void **)&tmpx, V * u->cin * 4) != cudaSuccess) return GNB_ENOMEM;
        cudaMemcpyAsync(tmpx, x, V * u->cin * 4, cudaMemcpyHostToDevice, u->s);
        xd = tmpx;
    }
    counted(k_pack_input)<<<(unsigned)((V + 255) / 256), 256, 0, u->s>>>(xd, u->cin, V, vox(u, 0, 1), u->xin);
    rc = unet_forward(u, batch);
    if (rc == GNB_OK)
        cudaMemcpyAsync(y, u->yout, V * u->cout * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        u->s);
    rc = unet_check(u, rc);
    if (tmpx) cudaFree(tmpx);
    return rc;
}

int gnb_unet_train_step(gnb_unet *u, int batch, const float *x, const float *target, double lr, double *loss,
                        int on_device)
{
    if (!u || !x || !target || batch < 1 || !(lr >= 0.0)) return GNB_EINVAL;
    int rc = unet_alloc_acts(u, batch);
    if (rc != GNB_OK) return rc;
    long long V = vox(u, 0, batch);
    float *tmpx = nullptr;
    const float *xd = x;
    if (!on_device) {
        if (cudaMalloc((void **)&tmpx, V * u->cin * 4) != cudaSuccess) return GNB_ENOMEM;
        cudaMemcpyAsync(tmpx, x, V * u->cin * 4, cudaMemcpyHostToDevice, u->s);
        xd = tmpx;
    }
    cudaMemcpyAsync(u->tgt, target, V * u->cout * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                    u->s);
    counted(k_pack_input)<<<(unsigned)((V + 255) / 256), 256, 0, u->s>>>(xd, u->cin, V, vox(u, 0, 1), u->xin);
    rc = unet_forward(u, batch);
    cudaMemsetAsync(u->loss_d, 0, 8, u->s);
    counted(k_mse)<<<(unsigned)((V * 16 + 255) / 256), 256, 0, u->s>>>(u->yout, u->tgt, V, vox(u, 0, 1), u->cout,
                                                                     u->dyb, u->loss_d);
    cudaMemsetAsync(u->g, 0, u->nparam * 4, u->s);
    if (rc == GNB_OK) rc = unet_backward(u, batch);
    if (rc == GNB_OK && lr > 0.0) {
        u->adam_t++;
        const double b1 = 0.9, b2 = 0.999;
        const double ic1 = 1.0 / (1.0 - std::pow(b1, (double)u->adam_t));
        const double ic2 = 1.0 / (1.0 - std::pow(b2, (double)u->adam_t));
        counted(k_adam)<<<(unsigned)((u->nparam + 255) / 256), 256, 0, u->s>>>(
            u->p, u->g, u->m, u->v, u->nparam, (float)lr, (float)b1, (float)(1.0 - b1), (float)b2, (float)(1.0 - b2),
            1e-8f, (float)ic1, (float)ic2);
        rc = unet_pack(u);
    }
    double l = 0.0;
    if (rc == GNB_OK) cudaMemcpyAsync(&l, u->loss_d, 8, cudaMemcpyDeviceToHost, u->s);
    rc = unet_check(u, rc);
    if (loss) *loss = l / (double)(V * u->cout);
    if (tmpx) cudaFree(tmpx);
    return rc;
}

}  // extern "C"
