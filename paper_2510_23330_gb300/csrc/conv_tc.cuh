// conv_tc.cuh -- host interface of the tcgen05 3^3 convolution (conv_tc.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace gnb {

constexpr unsigned TC_SMEM_MAX = 232448;  // opt-in dynamic shared memory per CTA (227 KB)
constexpr unsigned TC_SMEM_SM = 233472;   // shared memory per SM (228 KB)

// out[v][n] = act(bias[n] + sum_{tap, k} in[v + tap][k] * w[tap][k][n]) over the
// 27 taps of a zero-padded 3^3 neighbourhood; the input is the channel
// concatenation of in1 (C1 channels) and in2 (C2 channels), the output is
// split into out1 (channels [0, O1)) and out2 (channels [O1, N)).  All
// tensors are BF16 on a (B, D, H, W) grid, blocked by 8 channels:
// [B][C / 8][D][H][W][8]; C1, C2, O1 and N are multiples of 16.
struct TcConv {
    const __nv_bfloat16 *in1, *in2;
    int C1, C2;
    const __nv_bfloat16 *w;  // packed [27][(C1 + C2) / 8][N][8]
    const float *bias;       // [N] or null
    int N;
    __nv_bfloat16 *out1, *out2;
    int O1;
    int relu;
    int B, D, H, W;
    unsigned tx_extra;  // 0; > 0 only in the wait-timeout test (bytes the halo barrier expects beyond the loads)
    int plan;           // index into conv3_tc_plans' list (< 0 or out of range: the first, the rule's choice)
};

constexpr int TC_MAX_PLANS = 24;

struct TcPlan {
    int Zt, nbuf, wstages, dzn;
    unsigned plane, halo, off_w, off_h, wbytes, smem, tmem_cols;
};

// Tile depth, buffering and shared-memory layout for N output and K input
// channels on a grid of depth D: all 27 taps' weights resident when they fit,
// else a ring of 4 to 2 one-tap stages streamed per tile; false when the
// shape is not supported (N or K not a multiple of 16, N > 256, or not even a
// two-stage ring fits).
bool conv3_tc_plan(int N, int K, int D, TcPlan *pl);
// Every supported plan for the shape, the rule's choice first (at most cap);
// the number written.  The tile autotuner times them on the real layer.
int conv3_tc_plans(int N, int K, int D, TcPlan *out, int cap);

// Launches the convolution on s.  Returns 1 when launched, 0 when the shape
// or alignment is not supported (nothing launched; the caller uses another
// kernel), -1 when a supported shape cannot be launched (tensor-map encoding
// or launch error).  A device-side wait that runs out writes a
// non-zero code into *err (device memory).
int conv3_tc(const TcConv &c, int *err, cudaStream_t s);

// 2x2x2 transposed convolution with stride 2 (the U-Net's up-sampling) on
// the tensor cores: out(fine voxel 2 v + (dz, dy, dx))[n] = bias[n] +
// sum_k in(v)[k] w[t][k][n], t = 4 dz + 2 dy + dx, blocked BF16 tensors on a
// (B, Dc^3) coarse and (B, (2 Dc)^3) fine grid; w in the layout of pack_w_tc
// with taps = 1 and 8 N rows (row t N + n).  Returns 1 when launched, 0 when
// the shape is not supported (Dc^3 not a multiple of 128, N > 64, ...),
// -1 on a launch error.
bool up2_tc_ok(int N, int K, long long Vc);
int up2_tc(const __nv_bfloat16 *in, const __nv_bfloat16 *w, const float *bias, __nv_bfloat16 *out, int B, int Dc,
           int K, int N, int *err, cudaStream_t s);

// Weight gradient of a 3^3 "same" convolution, dw[t][c][n] += sum_v
// x(v + tap t)[c] g(v)[n] (FP32 atomics into dw, [27][Cw][N]), on the tensor
// cores; x is the concatenation of x1 (C1 channels) and x2 (C2), g has Cg
// channels (the first N used), blocked BF16 tensors on a (B, D^3) grid.
// Returns 1 when launched, 0 when the shape is not supported (C1 + C2 not
// in {16, 32, 64, 128}, N not a multiple of 16 in [16, 128], ...), -1 on a
// launch error.
int wgrad3_tc(const __nv_bfloat16 *x1, int C1, const __nv_bfloat16 *x2, int C2, const __nv_bfloat16 *g, int Cg, int N,
              int Cw, float *dw, int B, int D, int *err, cudaStream_t s);

// Whether a 3^3 layer with N output and K input channels runs with its
// three z-taps in one MMA (N <= 32; see conv_tc.cu).
bool conv3_tc_dzn(int N, int K);

// Re-layout of packed weights [taps][Npad][Kpad] into the tensor-core
// layout [taps][Kpad / 8][Npad][8], or, for the layers of conv3_tc_dzn,
// [9 (y, x)-taps][Kpad / 8][3 Npad (z-taps 2, 1, 0)][8].
int pack_w_tc(const __nv_bfloat16 *src, int taps, int Npad, int Kpad, __nv_bfloat16 *dst, cudaStream_t s);

}  // namespace gnb
