// conv_tc.cu -- 3^3 "same" convolution of BF16 NDHWC activations on the
// 5th-generation tensor cores (tcgen05 + TMEM), used for the forward pass and
// the input gradient of the surrogate U-Net's 3^3 convolutions (Sec. 3.3 of
// Hirashima et al., SC'25).
//
// Activations are blocked by 8 channels, [batch][channel / 8][z][y][x][8], so
// 10 x voxels of one channel group are one contiguous 160-byte row.
//
// One output tile is 8 (x) x 16 (y) voxels x Zt z-planes; each z-plane is one
// M = 128 MMA row block (row r = 8 y + x).  The tile's input halo,
// (Zt + 2) x 18 x 10 voxels, is brought into shared memory once by TMA (one
// 4-D box of 18 (Zt + 2) rows of 160 bytes per channel group; out-of-range
// voxels are zero-filled by the TMA unit, which is exactly the zero padding
// of the convolution) and lands as [channel group][z][y][x][8 channels]:
// eight consecutive x voxels of one channel group form one 8 x 16-byte core
// matrix of the canonical K-major no-swizzle layout, so every one of the 27
// taps is the same descriptor with its start address shifted by the tap's
// (z, y, x) offset -- no im2col copy.
// The weights of all taps stay resident in shared memory for the whole
// persistent CTA, packed [tap][channel group][N][8].
//
// Roles (192 threads): warp 4 lane 0 issues the TMA loads, warp 5 runs the
// MMA loop warp-uniformly and one elected lane issues tcgen05.mma (FP32
// accumulators in TMEM), warps 0..3 read TMEM with
// tcgen05.ld and apply bias, ReLU and the BF16 store.  Halo buffers and TMEM
// accumulators are double buffered so the loads of tile i + 1, the MMAs of
// tile i and the epilogue of tile i - 1 overlap.  Every mbarrier wait is
// bounded (1 s of %globaltimer); a wait that runs out sets the error word,
// all roles leave their loops, in-flight copies and MMAs are drained (again
// bounded) and TMEM is freed before the CTA exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "conv_tc.cuh"

typedef __nv_bfloat16 bf16;

namespace gnb {

namespace {

constexpr int TC_THREADS = 192;
constexpr int HX = 10, HY = 18;          // halo extent in x and y
constexpr unsigned ROW_BYTES = 16;       // one voxel of one 8-channel group
constexpr unsigned YSTRIDE = HX * ROW_BYTES;
constexpr unsigned ZSTRIDE = HY * YSTRIDE;
constexpr unsigned HDR = 256;            // barriers, TMEM slot, abort word
constexpr int MAX_WSTAGE = 4;            // weight ring stages when the weights are streamed
constexpr unsigned ALIGN_SLACK = 1024;
constexpr unsigned long long WAIT_NS = 1000000000ull;

enum { B_W = 0, B_HF = 1, B_HE = 3, B_AF = 5, B_AE = 7, B_DR = 9, B_WF = 10, B_WE = 14, NBARS = 18 };

struct TcArgs {
    const bf16 *w;
    const float *bias;
    bf16 *out1, *out2;
    int N, K, C1, O1, relu;
    int B, D, H, W;
    int Zt, nbuf, tx, ty, tz;
    int wstages;  // 0: all 27 taps resident; else a ring of this many one-tap stages
    int dzn;      // 1: the three z-taps share one MMA (N = 3 N_out, sliding TMEM windows)
    unsigned acc_cols;  // TMEM columns of one accumulator buffer
    long long ntiles;
    unsigned wbytes, plane, halo, off_w, off_h, tx_bytes, tmem_cols, idesc;
    int *err;
};

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mb_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mb_arrive(unsigned bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mb_try(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for the phase of `parity`.  Returns false when another role
// has aborted (honour_abort) or after WAIT_NS, in which case it aborts the
// CTA and records `code` in the error word.
__device__ bool mb_wait(unsigned bar, unsigned parity, volatile int *abort_flag, int *err, int code,
                        bool honour_abort = true)
{
    unsigned long long t0 = 0;
    for (unsigned it = 0;; it++) {
        if (mb_try(bar, parity)) return true;
        if (honour_abort && *abort_flag) return false;
        if ((it & 31u) == 0) {
            unsigned long long t = gtimer();
            if (t0 == 0) t0 = t;
            else if (t - t0 > WAIT_NS) {
                *abort_flag = 1;
                atomicExch(err, code);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_load_4d(unsigned dst, const CUtensorMap *m, int c0, int c1, int c2, int c3,
                                            unsigned bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];\n" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(m)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void bulk_load(unsigned dst, const void *src, unsigned bytes, unsigned bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// Shared-memory matrix descriptors, canonical K-major layout without swizzle:
// start address, leading-dimension byte offset (between core matrices along
// K), stride-dimension byte offset (between 8-row groups along M or N), and
// the descriptor version bit 46.  The low 32-bit word holds the start address
// in 16-byte units (bits 0-13) and the leading offset (bits 16-29), so moving
// the start by a multiple of 16 bytes is one add on the low word; the high
// word holds the stride offset and the version bit.
__device__ __forceinline__ unsigned sdesc_lo(unsigned addr, unsigned lbo)
{
    return ((addr & 0x3FFFFu) >> 4) | ((lbo >> 4) << 16);
}
__device__ __forceinline__ unsigned sdesc_hi(unsigned sbo) { return (sbo >> 4) | (1u << 14); }
__device__ __forceinline__ unsigned long long dpair(unsigned lo, unsigned hi)
{
    return ((unsigned long long)hi << 32) | lo;
}

// MMA and commit are executed by the whole warp in uniform control flow (so
// the operands stay warp-uniform); elect.sync picks the one lane that issues.
__device__ __forceinline__ void tc_mma_elect(unsigned d, unsigned long long a, unsigned long long b, unsigned idesc,
                                             unsigned acc)
{
    asm volatile(
        "{\n .reg .pred e, p;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 p, %4, 0;\n"
        " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tc_commit_elect(unsigned bar)
{
    asm volatile(
        "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
        " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(bar)
        : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane; the wait is in the
// same statement so no use of the registers can be scheduled before it.
__device__ __forceinline__ void tc_ld16(unsigned taddr, float *v)
{
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// 8 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld8(unsigned taddr, float *v)
{
    unsigned r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] = __uint_as_float(r[i]);
}

// Zeros 16 consecutive FP32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tc_st16_zero(unsigned taddr)
{
    const unsigned z = 0u;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
        "%1};\n" ::"r"(taddr),
        "r"(z)
        : "memory");
}
__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

__device__ __forceinline__ void decode_tile(const TcArgs &p, int Zt, long long t, int &bb, int &z0, int &y0, int &x0)
{
    int xt = (int)(t % p.tx);
    t /= p.tx;
    int yt = (int)(t % p.ty);
    t /= p.ty;
    int zt = (int)(t % p.tz);
    bb = (int)(t / p.tz);
    x0 = 8 * xt;
    y0 = 16 * yt;
    z0 = Zt * zt;
}

// The MMAs of one dz-in-N tile.  Input plane j, in-plane tap (ty, tx): one
// MMA of N = 3 N_out whose column window [j N, (j + 3) N) holds output planes
// j - 2, j - 1, j (z-taps 2, 1, 0); every MMA accumulates.  Windows of planes
// j = r, r + 3, ... are disjoint, so issuing them back to back keeps several
// accumulations in flight instead of a chain of dependent MMAs.  With the
// tile depth and K / 16 known at compile time the loop nest is straight-line
// code: a small-N MMA takes only ~40 cycles of the tensor core, and a loop
// with run-time bounds spends about twice that per MMA on issue.
template <int ZT, int NKS>
__device__ __forceinline__ void issue_dzn(const TcArgs &p, unsigned alo0, unsigned sW, unsigned d0)
{
    const int Zt = ZT ? ZT : p.Zt, nks = NKS ? NKS : (p.K >> 4);
    const unsigned ahi = sdesc_hi(YSTRIDE), bhi = sdesc_hi(128u);
    const unsigned zs4 = ZSTRIDE >> 4, pl4 = (2u * p.plane) >> 4;
    const unsigned n3 = 3u * (unsigned)p.N;
    const unsigned wyx4 = ((unsigned)nks * 2u * n3 * 16u) >> 4;  // one (ty, tx) slice of weights
    const unsigned bk4 = (2u * n3 * 16u) >> 4;
    const unsigned blo0 = sdesc_lo(sW, n3 * 16u);
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int yx = 0; yx < 9; yx++) {
            const unsigned aoff = ((unsigned)(yx / 3) * YSTRIDE + (unsigned)(yx % 3) * ROW_BYTES) >> 4;
#pragma unroll
            for (int ks = 0; ks < nks; ks++) {
                const unsigned long long bd = dpair(blo0 + (unsigned)yx * wyx4 + (unsigned)ks * bk4, bhi);
#pragma unroll
                for (int j = r; j < Zt + 2; j += 3)
                    tc_mma_elect(d0 + (unsigned)(j * p.N), dpair(alo0 + aoff + (unsigned)ks * pl4 + (unsigned)j * zs4, ahi),
                                 bd, p.idesc, 1u);
            }
        }
}

// DZ: 1 dz-in-N, 0 plain, -1 read from p; ZT: tile depth (0: read from p);
// NKS: K / 16 (0: read from p).
template <int DZ, int ZT, int NKS>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_conv3_tc(const __grid_constant__ CUtensorMap m1, const __grid_constant__ CUtensorMap m2, const TcArgs p)
{
    const int Zt = ZT ? ZT : p.Zt;
    const bool dzn = DZ >= 0 ? DZ != 0 : p.dzn != 0;
    extern __shared__ unsigned char dsm[];
    const unsigned raw = smem_u32(dsm);
    const unsigned sb = (raw + (ALIGN_SLACK - 1)) & ~(ALIGN_SLACK - 1);
    unsigned char *gb = dsm + (sb - raw);
    unsigned *slot = reinterpret_cast<unsigned *>(gb + 8 * NBARS);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(gb + 8 * NBARS + 4);
    const unsigned sW = sb + p.off_w, sH = sb + p.off_h;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    auto bar = [&](int i) { return sb + 8u * (unsigned)i; };

    if (threadIdx.x == 0) {
        mb_init(bar(B_W), 1);
        for (int b = 0; b < 2; b++) {
            mb_init(bar(B_HF + b), 1);
            mb_init(bar(B_HE + b), 1);
            mb_init(bar(B_AF + b), 1);
            mb_init(bar(B_AE + b), 128);
        }
        mb_init(bar(B_DR), 1);
        for (int q = 0; q < MAX_WSTAGE; q++) {
            mb_init(bar(B_WF + q), 1);
            mb_init(bar(B_WE + q), 1);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slot)),
                     "r"(p.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *slot;
    const int kc8 = p.K >> 3;
    if (dzn) {
        // the sliding accumulator windows start from zero: the epilogue warps
        // clear both buffers here and each buffer again after reading it
        if (warp < 4) {
            for (unsigned c = 0; c < (unsigned)p.nbuf * p.acc_cols; c += 16)
                tc_st16_zero(tmem + ((unsigned)(32 * warp) << 16) + c);
            tc_wait_st();
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }

    if (warp == 4) {
        if (lane == 0) {
            // ---------------------------------------------------------- producer
            const unsigned wtap = (unsigned)kc8 * (unsigned)p.N * 16u;  // bytes of one tap's weights
            if (!p.wstages) {
                mb_expect_tx(bar(B_W), p.wbytes);
                for (unsigned o = 0; o < p.wbytes; o += 32768u) {
                    unsigned n = p.wbytes - o < 32768u ? p.wbytes - o : 32768u;
                    bulk_load(sW + o, reinterpret_cast<const unsigned char *>(p.w) + o, n, bar(B_W));
                }
            }
            int uses[2] = {0, 0};
            long long wg = 0;  // weight-tap loads issued (streamed mode)
            bool stop = false;
            int i = 0;
            for (long long t = blockIdx.x; t < p.ntiles; t += gridDim.x, i++) {
                const int b = i % p.nbuf;
                const unsigned k = (unsigned)(i / p.nbuf);
                if (k > 0 && !mb_wait(bar(B_HE + b), (k - 1) & 1u, abort_flag, p.err, 1)) break;
                int bb, z0, y0, x0;
                decode_tile(p, Zt, t, bb, z0, y0, x0);
                mb_expect_tx(bar(B_HF + b), p.tx_bytes);
                const unsigned dst = sH + (unsigned)b * p.halo;
                // x and the 8 channels of a group form the innermost TMA
                // dimension: start 8 (x0 - 1) elements = 16 (x0 - 1) bytes
                const int g1 = p.C1 >> 3, g2 = (p.K - p.C1) >> 3;
                for (int kc = 0; kc < kc8; kc++) {
                    if (kc < g1)
                        tma_load_4d(dst + kc * p.plane, &m1, 8 * (x0 - 1), y0 - 1, z0 - 1, bb * g1 + kc, bar(B_HF + b));
                    else
                        tma_load_4d(dst + kc * p.plane, &m2, 8 * (x0 - 1), y0 - 1, z0 - 1, bb * g2 + (kc - g1),
                                    bar(B_HF + b));
                }
                uses[b]++;
                // streamed weights: the 27 taps of this tile through the ring
                for (int tap = 0; p.wstages && tap < 27; tap++, wg++) {
                    const int st = (int)(wg % p.wstages);
                    const unsigned kk = (unsigned)(wg / p.wstages);
                    if (kk > 0 && !mb_wait(bar(B_WE + st), (kk - 1) & 1u, abort_flag, p.err, 8)) {
                        stop = true;
                        break;
                    }
                    mb_expect_tx(bar(B_WF + st), wtap);
                    bulk_load(sW + (unsigned)st * wtap, reinterpret_cast<const unsigned char *>(p.w) + (size_t)tap * wtap,
                              wtap, bar(B_WF + st));
                }
                if (stop) break;
            }
            // drain: every copy this CTA issued has landed before it exits
            if (!p.wstages) mb_wait(bar(B_W), 0, abort_flag, p.err, 2, false);
            for (int b = 0; b < 2; b++)
                if (uses[b] > 0) mb_wait(bar(B_HF + b), (unsigned)(uses[b] - 1) & 1u, abort_flag, p.err, 2, false);
            for (int st = 0; p.wstages && st < p.wstages; st++) {
                // the last load issued into stage st is number (wg - 1 - ((wg - 1 - st) mod S))
                if (wg > st) {
                    const long long last = st + ((wg - 1 - st) / p.wstages) * p.wstages;
                    mb_wait(bar(B_WF + st), (unsigned)(last / p.wstages) & 1u, abort_flag, p.err, 2, false);
                }
            }
        }
    } else if (warp == 5) {
        // ------------------------------------------------------------------ MMA
        // The Zt z-planes of a tile accumulate into Zt independent TMEM
        // blocks; their MMAs are interleaved so consecutive MMAs never feed
        // the same accumulator.
        int ok = p.wstages ? 1 : mb_wait(bar(B_W), 0, abort_flag, p.err, 3);
        if (__all_sync(0xffffffffu, ok)) {
            long long wg = 0;  // weight taps consumed (streamed mode)
            const unsigned wtap = (unsigned)kc8 * (unsigned)p.N * 16u;  // bytes of one tap's weights
            const unsigned nbytes16 = (unsigned)p.N * 16u;              // one channel group of weights
            int i = 0;
            for (long long t = blockIdx.x; t < p.ntiles; t += gridDim.x, i++) {
                const int b = i % p.nbuf;
                const unsigned k = (unsigned)(i / p.nbuf);
                ok = mb_wait(bar(B_HF + b), k & 1u, abort_flag, p.err, 4);
                if (!__all_sync(0xffffffffu, ok)) break;
                if (k > 0) {
                    ok = mb_wait(bar(B_AE + b), (k - 1) & 1u, abort_flag, p.err, 5);
                    if (!__all_sync(0xffffffffu, ok)) break;
                }
                tc_fence_after();
                const unsigned hb = sH + (unsigned)b * p.halo;
                const unsigned d0 = tmem + (unsigned)b * p.acc_cols;
                bool stop = false;
                // descriptors are stepped as 32-bit low words (start address in
                // 16-byte units): a few adds per MMA
                const unsigned ahi = sdesc_hi(YSTRIDE), bhi = sdesc_hi(128u);
                const unsigned alo0 = sdesc_lo(hb, p.plane);
                const unsigned zs4 = ZSTRIDE >> 4, pl4 = (2u * p.plane) >> 4;
                if (dzn) issue_dzn<ZT, NKS>(p, alo0, sW, d0);
                const unsigned nb4 = (2u * (unsigned)p.N * 16u) >> 4;  // two channel groups of weights
                for (int tap = 0; !dzn && tap < 27; tap++) {
                    const int tz = tap / 9, ty = (tap / 3) % 3, tx = tap % 3;
                    unsigned alo = alo0 + (((unsigned)tz * ZSTRIDE + (unsigned)ty * YSTRIDE + (unsigned)tx * ROW_BYTES) >> 4);
                    unsigned w0 = sW + (unsigned)tap * wtap;
                    int st = 0;
                    if (p.wstages) {
                        st = (int)(wg % p.wstages);
                        ok = mb_wait(bar(B_WF + st), (unsigned)(wg / p.wstages) & 1u, abort_flag, p.err, 9);
                        if (!__all_sync(0xffffffffu, ok)) { stop = true; break; }
                        tc_fence_after();
                        w0 = sW + (unsigned)st * wtap;
                    }
                    unsigned blo = sdesc_lo(w0, nbytes16);
                    for (int ks = 0; ks < (p.K >> 4); ks++, alo += pl4, blo += nb4) {
                        const unsigned long long bd = dpair(blo, bhi);
                        const unsigned acc = (tap | ks) != 0;
#pragma unroll
                        for (int zz = 0; zz < Zt; zz++)
                            tc_mma_elect(d0 + (unsigned)(zz * p.N), dpair(alo + (unsigned)zz * zs4, ahi), bd, p.idesc, acc);
                    }
                    if (p.wstages) {
                        tc_commit_elect(bar(B_WE + st));  // the stage is free once these MMAs complete
                        wg++;
                    }
                }
                if (stop) break;
                tc_commit_elect(bar(B_HE + b));
                tc_commit_elect(bar(B_AF + b));
            }
        }
        // drain: all MMAs issued by this warp's elected lane are complete
        tc_commit_elect(bar(B_DR));
        mb_wait(bar(B_DR), 0, abort_flag, p.err, 6, false);
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        const int r = 32 * warp + lane;  // TMEM lane = row of the M = 128 block
        const unsigned lane_addr = (unsigned)(32 * warp) << 16;
        const long long Vs = (long long)p.D * p.H * p.W;
        int i = 0;
        for (long long t = blockIdx.x; t < p.ntiles; t += gridDim.x, i++) {
            const int b = i % p.nbuf;
            const unsigned k = (unsigned)(i / p.nbuf);
            int ok = mb_wait(bar(B_AF + b), k & 1u, abort_flag, p.err, 7);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            tc_fence_after();
            int bb, z0, y0, x0;
            decode_tile(p, Zt, t, bb, z0, y0, x0);
            const int x = x0 + (r & 7), y = y0 + (r >> 3);
            for (int zz = 0; zz < Zt; zz++) {
                const int z = z0 + zz;
                const bool valid = x < p.W && y < p.H && z < p.D;
                const long long sv = ((long long)z * p.H + y) * p.W + x;
                for (int c0 = 0; c0 < p.N; c0 += 16) {
                    float f[16];
                    __syncwarp();
                    tc_ld16(tmem + lane_addr + (unsigned)b * p.acc_cols + (unsigned)((zz + (dzn ? 2 : 0)) * p.N + c0),
                            f);
                    if (!valid) continue;
                    if (p.bias) {
#pragma unroll
                        for (int q = 0; q < 16; q++) f[q] += __ldg(p.bias + c0 + q);
                    }
                    if (p.relu) {
#pragma unroll
                        for (int q = 0; q < 16; q++) f[q] = fmaxf(f[q], 0.f);
                    }
                    uint4 o[2];
                    unsigned *ou = reinterpret_cast<unsigned *>(o);
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        __nv_bfloat162 h2 = __floats2bfloat162_rn(f[2 * q], f[2 * q + 1]);
                        ou[q] = *reinterpret_cast<unsigned *>(&h2);
                    }
                    // two channel groups: two 16-byte pieces, Vs * 8 elements apart
                    const bool lo = c0 < p.O1;
                    const int Cx = lo ? p.O1 : p.N - p.O1, cc = lo ? c0 : c0 - p.O1;
                    bf16 *dst = (lo ? p.out1 : p.out2) + (((long long)bb * (Cx >> 3) + (cc >> 3)) * Vs + sv) * 8;
                    *reinterpret_cast<uint4 *>(dst) = o[0];
                    *reinterpret_cast<uint4 *>(dst + Vs * 8) = o[1];
                }
            }
            if (dzn) {
                __syncwarp();
                for (unsigned c = 0; c < p.acc_cols; c += 16) tc_st16_zero(tmem + lane_addr + (unsigned)b * p.acc_cols + c);
                tc_wait_st();
            }
            tc_fence_before();
            mb_arrive(bar(B_AE + b));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 4) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(p.tmem_cols)
                     : "memory");
    }
}

typedef CUresult (*encode_fn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

encode_fn get_encode()
{
    static encode_fn fn = []() -> encode_fn {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<encode_fn>(f);
    }();
    return fn;
}

// Tensor map of a blocked BF16 tensor [B][C / 8][D][H][W][8] viewed as 4-D
// (8 W, H, D, B C / 8) and read in halo boxes of 8 x 10 elements (10 voxels
// of one channel group) x 18 x zh.
bool make_map(CUtensorMap *m, const bf16 *ptr, int C, int B, int D, int H, int W, int zh)
{
    encode_fn enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[4] = {(cuuint64_t)W * 8, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)B * (C / 8)};
    cuuint64_t strides[3] = {(cuuint64_t)W * 16, (cuuint64_t)H * W * 16, (cuuint64_t)D * H * W * 16};
    cuuint32_t box[4] = {8 * HX, (cuuint32_t)HY, (cuuint32_t)zh, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16 *>(ptr), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int device_sms()
{
    static int n = []() {
        int d = 0, v = 0;
        cudaGetDevice(&d);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d);
        return v > 0 ? v : 1;
    }();
    return n;
}

unsigned pow2_at_least(unsigned v)
{
    unsigned c = 32;
    while (c < v) c <<= 1;
    return c;
}


// ------------------------------------------------------------------ UP2
// 2x2x2 transposed convolution with stride 2 on the tensor cores: one tile is
// 128 consecutive coarse voxels of one batch entry (M = 128) and all eight
// taps' output channels form N = 8 N_out, so a tile is K / 16 MMAs (split in
// two when 8 N_out > 256).  In the blocked layout the 128 voxels of one
// channel group are 2 KB of contiguous memory, i.e. exactly a column of
// K-major core matrices; the tile and the weights arrive by bulk copies.
struct Up2Args {
    const bf16 *in;      // coarse [B][K / 8][Vc][8]
    const bf16 *w;       // [K / 8][8 N][8], row t N + n = tap t, output channel n
    const float *bias;   // [N] or null
    bf16 *out;           // fine [B][N / 8][8 Vc][8]
    int K, N, Dc;        // input channels, output channels, coarse grid edge
    long long Vc, ntiles;
    unsigned abytes, wbytes, tmem_cols, idesc, nsplit, ncols_split;
    int *err;
};
constexpr unsigned UP_HDR = 256;

__global__ void __launch_bounds__(128) k_up2_tc(const Up2Args p)
{
    extern __shared__ unsigned char dsm[];
    const unsigned raw = smem_u32(dsm);
    const unsigned sb = (raw + (ALIGN_SLACK - 1)) & ~(ALIGN_SLACK - 1);
    unsigned char *gb = dsm + (sb - raw);
    unsigned *slot = reinterpret_cast<unsigned *>(gb + 16);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(gb + 20);
    const unsigned bar_ld = sb, bar_mma = sb + 8;
    const unsigned sA = sb + UP_HDR, sB = sA + p.abytes;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long r0 = (long long)blockIdx.x * 128;
    const long long bb = r0 / p.Vc, v0 = r0 - bb * p.Vc;
    const int kc8 = p.K >> 3;
    if (threadIdx.x == 0) {
        mb_init(bar_ld, 1);
        mb_init(bar_mma, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slot)),
                     "r"(p.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *slot;
    if (threadIdx.x == 0) {
        mb_expect_tx(bar_ld, p.abytes + p.wbytes);
        for (int kc = 0; kc < kc8; kc++)
            bulk_load(sA + (unsigned)kc * 2048u, p.in + ((bb * kc8 + kc) * p.Vc + v0) * 8, 2048u, bar_ld);
        for (unsigned o = 0; o < p.wbytes; o += 32768u) {
            unsigned n = p.wbytes - o < 32768u ? p.wbytes - o : 32768u;
            bulk_load(sB + o, reinterpret_cast<const unsigned char *>(p.w) + o, n, bar_ld);
        }
    }
    bool ok = true;
    if (warp == 1) {
        ok = __all_sync(0xffffffffu, mb_wait(bar_ld, 0, abort_flag, p.err, 11));
        if (ok) {
            tc_fence_after();
            const unsigned ahi = sdesc_hi(128u), bhi = sdesc_hi(128u);
            const unsigned nrow16 = (unsigned)(8 * p.N) * 16u;  // one channel group of all weight rows
            for (int ks = 0; ks < (p.K >> 4); ks++)
                for (unsigned h = 0; h < p.nsplit; h++)
                    tc_mma_elect(tmem + h * p.ncols_split,
                                 dpair(sdesc_lo(sA + (unsigned)ks * 4096u, 2048u), ahi),
                                 dpair(sdesc_lo(sB + (unsigned)ks * 2u * nrow16 + h * p.ncols_split * 16u, nrow16), bhi),
                                 p.idesc, ks != 0);
            tc_commit_elect(bar_mma);
        }
    }
    // every thread: the accumulators are ready (or the CTA gave up)
    ok = mb_wait(bar_mma, 0, abort_flag, p.err, 12);
    ok = __all_sync(0xffffffffu, ok);
    if (ok) {
        tc_fence_after();
        const int r = 32 * warp + lane;
        const unsigned lane_addr = (unsigned)(32 * warp) << 16;
        const long long v = v0 + r;
        const int D = p.Dc, x = (int)(v % D), y = (int)((v / D) % D), z = (int)(v / ((long long)D * D));
        const long long Vf = 8 * p.Vc;
        const int F = 2 * D;
        // taps in pairs (dx = 0, 1): the two fine voxels are adjacent in x,
        // so each channel group is one 32-byte store
        for (int tp = 0; tp < 4; tp++) {
            const int dz = tp >> 1, dy = tp & 1;
            const long long fv = ((long long)(2 * z + dz) * F + (2 * y + dy)) * F + 2 * x;
            for (int g = 0; g < (p.N >> 3); g++) {
                float f0[16], f1[16];
                // columns of tap (dz, dy, 0) and (dz, dy, 1): t N + 8 g + j
                const unsigned c0 = (unsigned)((2 * tp) * p.N + 8 * g), c1 = c0 + (unsigned)p.N;
                __syncwarp();
                tc_ld8(tmem + lane_addr + c0, f0);
                tc_ld8(tmem + lane_addr + c1, f1);
                uint4 o[2];
                unsigned *ou = reinterpret_cast<unsigned *>(o);
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const float b0 = p.bias ? __ldg(p.bias + 8 * g + 2 * q) : 0.f;
                    const float b1 = p.bias ? __ldg(p.bias + 8 * g + 2 * q + 1) : 0.f;
                    __nv_bfloat162 h0 = __floats2bfloat162_rn(f0[2 * q] + b0, f0[2 * q + 1] + b1);
                    __nv_bfloat162 h1 = __floats2bfloat162_rn(f1[2 * q] + b0, f1[2 * q + 1] + b1);
                    ou[q] = *reinterpret_cast<unsigned *>(&h0);
                    ou[4 + q] = *reinterpret_cast<unsigned *>(&h1);
                }
                bf16 *dst = p.out + ((bb * (p.N >> 3) + g) * Vf + fv) * 8;
                reinterpret_cast<uint4 *>(dst)[0] = o[0];
                reinterpret_cast<uint4 *>(dst)[1] = o[1];
            }
        }
    }
    if (threadIdx.x == 0) mb_wait(bar_ld, 0, abort_flag, p.err, 13, false);  // no copy outlives the CTA
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(p.tmem_cols)
                     : "memory");
    }
}


// ------------------------------------------------------------------ WGRAD
// Weight gradient of a 3^3 "same" convolution on the tensor cores:
//   dW[t][c][n] = sum_v x(v + tap t)[c] * g(v)[n]
// as a GEMM whose M = 128 rows are (tap slot s, input channel c) pairs --
// 128 / C taps of one tap group side by side, so every row is a real weight
// even for C = 16 -- whose N columns are the output channels and whose K is
// the voxels.  A CTA takes one tap group and one chunk of voxels; per stage of
// 64 voxels the threads gather the shifted inputs and the output gradient
// (zero outside the grid) and write them transposed into the canonical
// K-major core-matrix layout (8 rows x 16 bytes, rows = channels, the 16
// bytes = 8 voxels), one elected lane issues four K = 16 MMAs into a TMEM
// accumulator, and the stage buffers are double buffered behind the MMAs'
// commit barriers.  At the end each warp reads its 32 TMEM lanes (rows) and
// adds them to dW with FP32 atomics (the voxel chunks are split-K).
struct WgTcArgs {
    const bf16 *x1, *x2;   // input channels [0, C1) from x1, [C1, C) from x2; blocked [B][C/8][V][8]
    int C1, C;
    const bf16 *g;         // output gradient, blocked with Cg channels
    int Cg, N, Cw;         // channels of g, output channels of dW, input channels of dW (<= C)
    float *dw;             // [27][Cw][N]
    int B, D;              // grid (cube of edge D) and batch
    int ntap;              // taps per group: 128 / C
    long long V, chunk;    // voxels in all, voxels per CTA (multiple of 64)
    int nchunk;
    unsigned tmem_cols, idesc, abytes, bbytes;
    int *err;
};
constexpr unsigned WG_HDR = 256;
constexpr int WG_VS = 64;  // voxels per stage

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// offset of (row r, voxel k) in a K-major stage of WG_VS voxels whose M (or N)
// has rows rows: [k / 16][r / 8][(k % 16) / 8][r % 8][k % 8]
__device__ __forceinline__ unsigned wg_off(int r, int k, int rows)
{
    return (unsigned)(k >> 4) * (unsigned)rows * 32u + (unsigned)(r >> 3) * 256u + (unsigned)((k >> 3) & 1) * 128u +
           (unsigned)(r & 7) * 16u + (unsigned)(k & 7) * 2u;
}

__global__ void __launch_bounds__(128) k_wgrad_tc(const WgTcArgs p)
{
    extern __shared__ unsigned char dsm[];
    const unsigned raw = smem_u32(dsm);
    const unsigned sb = (raw + (ALIGN_SLACK - 1)) & ~(ALIGN_SLACK - 1);
    unsigned char *gb = dsm + (sb - raw);
    unsigned *slot = reinterpret_cast<unsigned *>(gb + 16);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(gb + 20);
    const unsigned bar0 = sb, bar1 = sb + 8;  // commit barriers of the two stage buffers
    const unsigned stage_bytes = p.abytes + p.bbytes;
    unsigned char *stg = gb + WG_HDR;
    const unsigned sStg = sb + WG_HDR;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tg = blockIdx.y;                // tap group
    const int t0 = tg * p.ntap;
    const int ntap = min(p.ntap, 27 - t0);
    const long long r0 = (long long)blockIdx.x * p.chunk, r1 = min(p.V, r0 + p.chunk);
    const int nstage = (int)((r1 - r0 + WG_VS - 1) / WG_VS);
    const long long D = p.D, Vs = D * D * D;
    if (tid == 0) {
        mb_init(bar0, 1);
        mb_init(bar1, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slot)),
                     "r"(p.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *slot;
    // rows of tap slots beyond ntap (a short last group) stay zero: cleared once
    for (unsigned o = (unsigned)tid * 16u; o < 2u * stage_bytes; o += 128u * 16u)
        *reinterpret_cast<uint4 *>(stg + o) = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    const int cg8 = p.C >> 3, ng8 = p.N >> 3;
    bool ok = true;
    int issued = -1;  // the last stage whose MMAs were issued
    for (int st = 0; st < nstage && ok; st++) {
        const int b = st & 1;
        const unsigned bar = b ? bar1 : bar0;
        // the MMAs that read this buffer two stages ago have finished
        if (st >= 2) ok = __syncthreads_and(mb_wait(bar, (unsigned)(((st - 2) >> 1) & 1), abort_flag, p.err, 21));
        if (!ok) break;
        unsigned char *sA = stg + (size_t)b * stage_bytes;
        unsigned char *sB = sA + p.abytes;
        const long long vb = r0 + (long long)st * WG_VS;
        // A: (tap slot, channel group, voxel) pieces of 8 channels
        for (int e = tid; e < ntap * cg8 * WG_VS; e += 128) {
            const int k = e % WG_VS, q = e / WG_VS;
            const int cg = q % cg8, s = q / cg8;
            const long long v = vb + k;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (v < r1) {
                const long long bb = v / Vs, rem = v - bb * Vs;
                const long long x = rem % D, y = (rem / D) % D, z = rem / (D * D);
                const int t = t0 + s;
                const long long zz = z + (t / 9 - 1), yy = y + ((t / 3) % 3 - 1), xx = x + (t % 3 - 1);
                if (zz >= 0 && zz < D && yy >= 0 && yy < D && xx >= 0 && xx < D) {
                    const long long src = (zz * D + yy) * D + xx;
                    const int c = cg * 8;
                    val = c < p.C1 ? *reinterpret_cast<const uint4 *>(p.x1 + ((bb * (p.C1 >> 3) + cg) * Vs + src) * 8)
                                   : *reinterpret_cast<const uint4 *>(
                                         p.x2 + ((bb * ((p.C - p.C1) >> 3) + (cg - (p.C1 >> 3))) * Vs + src) * 8);
                }
            }
            const unsigned short *h = reinterpret_cast<const unsigned short *>(&val);
            const int r = s * p.C + cg * 8;
#pragma unroll
            for (int j = 0; j < 8; j++) *reinterpret_cast<unsigned short *>(sA + wg_off(r + j, k, 128)) = h[j];
        }
        // B: (output channel group, voxel) pieces
        for (int e = tid; e < ng8 * WG_VS; e += 128) {
            const int k = e % WG_VS, ng = e / WG_VS;
            const long long v = vb + k;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (v < r1) {
                const long long bb = v / Vs, rem = v - bb * Vs;
                val = *reinterpret_cast<const uint4 *>(p.g + ((bb * (p.Cg >> 3) + ng) * Vs + rem) * 8);
            }
            const unsigned short *h = reinterpret_cast<const unsigned short *>(&val);
#pragma unroll
            for (int j = 0; j < 8; j++) *reinterpret_cast<unsigned short *>(sB + wg_off(ng * 8 + j, k, p.N)) = h[j];
        }
        fence_proxy_async_smem();  // the generic-proxy stores become visible to the tensor cores
        tc_fence_before();
        __syncthreads();
        if (warp == 0) {
            tc_fence_after();
            const unsigned a0 = sStg + (unsigned)b * stage_bytes, b0 = a0 + p.abytes;
            const unsigned hi = sdesc_hi(256u);
#pragma unroll
            for (int ks = 0; ks < WG_VS / 16; ks++)
                tc_mma_elect(tmem, dpair(sdesc_lo(a0 + (unsigned)ks * 128u * 32u, 128u), hi),
                             dpair(sdesc_lo(b0 + (unsigned)ks * (unsigned)p.N * 32u, 128u), hi), p.idesc,
                             (st > 0 || ks > 0) ? 1u : 0u);
            tc_commit_elect(bar);
        }
        issued = st;
    }
    // the last stage's MMAs (every commit of a barrier before it completed in order)
    if (ok && nstage > 0) {
        const int sl = nstage - 1;
        ok = __all_sync(0xffffffffu, mb_wait((sl & 1) ? bar1 : bar0, (unsigned)((sl >> 1) & 1), abort_flag, p.err, 22));
        ok = __syncthreads_and(ok);
    }
    if (ok && nstage > 0) {
        tc_fence_after();
        const int r = 32 * warp + lane;
        const int s = r / p.C, c = r - s * p.C;
        const bool live = s < ntap && c < p.Cw;
        const unsigned lane_addr = (unsigned)(32 * warp) << 16;
        for (int n0 = 0; n0 < p.N; n0 += 16) {
            float v[16];
            __syncwarp();
            tc_ld16(tmem + lane_addr + (unsigned)n0, v);
            if (live) {
                float *d = p.dw + ((long long)(t0 + s) * p.Cw + c) * p.N + n0;
#pragma unroll
                for (int j = 0; j < 16; j++) atomicAdd(d + j, v[j]);
            }
        }
    }
    if (!ok && issued >= 0 && tid == 0)  // no MMA outlives the CTA: its last commit covers the earlier ones
        mb_wait((issued & 1) ? bar1 : bar0, (unsigned)((issued >> 1) & 1), abort_flag, p.err, 23, false);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(p.tmem_cols)
                     : "memory");
    }
}

}  // namespace

// z-taps in N for the thin layers, which are otherwise bound by the
// shared-memory reads of A: when N <= 32 and the resident weights fit beside
// two halo buffers of two-plane tiles.
static bool dzn_fits(int N, int K, int zt, int nbuf, unsigned *smem, unsigned *cols, unsigned *plane,
                     unsigned *halo, unsigned *off_h)
{
    const unsigned wbytes = 27u * (unsigned)N * (unsigned)K * 2u;
    *plane = ((unsigned)(zt + 2) * ZSTRIDE + 127u) & ~127u;
    *halo = (unsigned)(K / 8) * *plane;
    *off_h = (HDR + wbytes + 127u) & ~127u;
    *smem = ALIGN_SLACK + *off_h + (unsigned)nbuf * *halo;
    const unsigned acc = (unsigned)((zt + 4) * N);
    *cols = pow2_at_least((unsigned)nbuf * acc);
    return *smem <= TC_SMEM_MAX && *cols <= 512;
}

bool conv3_tc_dzn(int N, int K)
{
    unsigned a, b, c, d, e;
    return N >= 16 && N <= 32 && (N % 16) == 0 && K >= 16 && (K % 16) == 0 && dzn_fits(N, K, 2, 2, &a, &b, &c, &d, &e);
}

int conv3_tc_plans(int N, int K, int D, TcPlan *out, int cap)
{
    if (N < 16 || N > 256 || (N % 16) || K < 16 || (K % 16) || cap < 1) return 0;
    int np = 0;
    if (conv3_tc_dzn(N, K)) {
        // the weights are packed for the dz-in-N MMA: only such plans apply
        static const int zd[] = {8, 4, 2};
        const int nbuf = 2;
        for (int zt : zd) {
            if (zt > 2 && zt > D) continue;
            unsigned smem, cols, plane, halo, off_h;
            if (!dzn_fits(N, K, zt, nbuf, &smem, &cols, &plane, &halo, &off_h)) continue;
            TcPlan &pl = out[np];
            pl.Zt = zt;
            pl.nbuf = nbuf;
            pl.wstages = 0;
            pl.dzn = 1;
            pl.plane = plane;
            pl.halo = halo;
            pl.off_w = HDR;
            pl.off_h = off_h;
            pl.wbytes = 27u * (unsigned)N * (unsigned)K * 2u;
            pl.smem = smem;
            pl.tmem_cols = cols;
            if (++np == cap) return np;
        }
        return np;
    }
    const unsigned wtap = (unsigned)N * (unsigned)K * 2u;
    static const int zts[] = {4, 2, 1};
    // resident weights first (even single-buffered: streaming the weights
    // costs more than the lost overlap); then a ring of 4, 3, 2 one-tap stages
    for (int stages = 0; stages <= MAX_WSTAGE; stages = stages ? stages - 1 : MAX_WSTAGE) {
        if (stages == 1) break;
        const unsigned wbytes = (stages ? (unsigned)stages : 27u) * wtap;
        for (int nbuf = 2; nbuf >= 1; nbuf--) {
            for (int zt : zts) {
                if (zt > 1 && zt > D) continue;
                const unsigned plane = ((unsigned)(zt + 2) * ZSTRIDE + 127u) & ~127u;
                const unsigned halo = (unsigned)(K / 8) * plane;
                const unsigned off_w = HDR;
                const unsigned off_h = (off_w + wbytes + 127u) & ~127u;
                const unsigned smem = ALIGN_SLACK + off_h + (unsigned)nbuf * halo;
                const unsigned cols = pow2_at_least((unsigned)(nbuf * zt * N));
                if (smem > TC_SMEM_MAX || cols > 512) continue;
                TcPlan &pl = out[np];
                pl.Zt = zt;
                pl.nbuf = nbuf;
                pl.wstages = stages;
                pl.dzn = 0;
                pl.plane = plane;
                pl.halo = halo;
                pl.off_w = off_w;
                pl.off_h = off_h;
                pl.wbytes = wbytes;
                pl.smem = smem;
                pl.tmem_cols = cols;
                if (++np == cap) return np;
            }
        }
    }
    return np;
}

bool conv3_tc_plan(int N, int K, int D, TcPlan *pl)
{
    return conv3_tc_plans(N, K, D, pl, 1) == 1;
}

using TcKernel = void (*)(const CUtensorMap, const CUtensorMap, const TcArgs);

// The instantiations: the hot tile shapes with compile-time loop bounds, and
// one run-time variant per mode for the rest.
const TcKernel TC_KERNELS[] = {k_conv3_tc<1, 8, 1>, k_conv3_tc<1, 4, 1>, k_conv3_tc<1, 4, 2>, k_conv3_tc<1, 0, 0>,
                               k_conv3_tc<0, 4, 0>, k_conv3_tc<0, 2, 0>, k_conv3_tc<0, 1, 0>, k_conv3_tc<0, 0, 0>};

TcKernel pick_kernel(const TcPlan &pl, int K)
{
    const int nks = K >> 4;
    if (pl.dzn) {
        if (pl.Zt == 8 && nks == 1) return TC_KERNELS[0];
        if (pl.Zt == 4 && nks == 1) return TC_KERNELS[1];
        if (pl.Zt == 4 && nks == 2) return TC_KERNELS[2];
        return TC_KERNELS[3];
    }
    if (pl.Zt == 4) return TC_KERNELS[4];
    if (pl.Zt == 2) return TC_KERNELS[5];
    if (pl.Zt == 1) return TC_KERNELS[6];
    return TC_KERNELS[7];
}

int conv3_tc(const TcConv &c, int *err, cudaStream_t s)
{
    const int K = c.C1 + c.C2, N = c.N;
    TcPlan plans[TC_MAX_PLANS];
    const int np = conv3_tc_plans(N, K, c.D, plans, TC_MAX_PLANS);
    if ((c.C1 % 8) || (c.C2 % 8) || (c.O1 % 16) || c.O1 > N || np < 1) return 0;
    const TcPlan pl = plans[c.plan >= 0 && c.plan < np ? c.plan : 0];
    if ((reinterpret_cast<uintptr_t>(c.w) & 15) || (reinterpret_cast<uintptr_t>(c.in1) & 15) ||
        (c.C2 && (reinterpret_cast<uintptr_t>(c.in2) & 15)))
        return 0;
    // from here on the shape is supported: a failure is an error, not a fallback
    CUtensorMap m1, m2;
    const int zh = pl.Zt + 2;
    if (!make_map(&m1, c.in1, c.C1, c.B, c.D, c.H, c.W, zh)) return -1;
    if (c.C2 > 0) {
        if (!make_map(&m2, c.in2, c.C2, c.B, c.D, c.H, c.W, zh)) return -1;
    } else {
        m2 = m1;
    }
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, []() {
        for (TcKernel k : TC_KERNELS) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM_MAX);
            if (e != cudaSuccess) attr_err = e;
        }
    });
    if (attr_err != cudaSuccess) return -1;
    TcArgs a;
    a.w = c.w;
    a.bias = c.bias;
    a.out1 = c.out1;
    a.out2 = c.out2 ? c.out2 : c.out1;
    a.N = N;
    a.K = K;
    a.C1 = c.C1;
    a.O1 = c.O1;
    a.relu = c.relu;
    a.B = c.B; a.D = c.D; a.H = c.H; a.W = c.W;
    a.Zt = pl.Zt;
    a.nbuf = pl.nbuf;
    a.wstages = pl.wstages;
    a.dzn = pl.dzn;
    a.acc_cols = (unsigned)((pl.dzn ? pl.Zt + 4 : pl.Zt) * N);
    a.tx = (c.W + 7) / 8;
    a.ty = (c.H + 15) / 16;
    a.tz = (c.D + pl.Zt - 1) / pl.Zt;
    a.ntiles = (long long)a.tx * a.ty * a.tz * c.B;
    a.wbytes = pl.wbytes;
    a.plane = pl.plane;
    a.halo = pl.halo;
    a.off_w = pl.off_w;
    a.off_h = pl.off_h;
    a.tx_bytes = (unsigned)(K / 8) * (unsigned)zh * ZSTRIDE + c.tx_extra;
    a.tmem_cols = pl.tmem_cols;
    // kind::f16 instruction descriptor: FP32 accumulator (bit 4), BF16 A
    // (bits 7-9 = 1) and B (bits 10-12 = 1), both K-major, N >> 3 at bit 17,
    // M >> 4 at bit 24 (M = 128).
    const int nmma = pl.dzn ? 3 * N : N;
    a.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(nmma >> 3) << 17) | ((128u >> 4) << 24);
    a.err = err;
    const int per_sm_smem = (int)(TC_SMEM_SM / (pl.smem + 1024u));
    const int per_sm_tmem = (int)(512u / pl.tmem_cols);
    int per_sm = per_sm_smem < per_sm_tmem ? per_sm_smem : per_sm_tmem;
    if (per_sm < 1) per_sm = 1;
    long long grid = (long long)device_sms() * per_sm;
    if (grid > a.ntiles) grid = a.ntiles;
    if (grid < 1) return 1;
    counted(pick_kernel(pl, K))<<<(unsigned)grid, TC_THREADS, pl.smem, s>>>(m1, m2, a);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

bool up2_tc_ok(int N, int K, long long Vc)
{
    return N >= 8 && N % 8 == 0 && 8 * N <= 512 && K >= 16 && K % 16 == 0 && Vc % 128 == 0 &&
           UP_HDR + ALIGN_SLACK + (unsigned)K / 8u * 2048u + (unsigned)K * 16u * (unsigned)N <= TC_SMEM_MAX;
}

int up2_tc(const bf16 *in, const bf16 *w, const float *bias, bf16 *out, int B, int Dc, int K, int N, int *err,
           cudaStream_t s)
{
    const long long Vc = (long long)Dc * Dc * Dc;
    if (!up2_tc_ok(N, K, Vc) || (reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(w) & 15) ||
        (reinterpret_cast<uintptr_t>(out) & 15))
        return 0;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, []() {
        attr_err = cudaFuncSetAttribute(k_up2_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM_MAX);
    });
    if (attr_err != cudaSuccess) return -1;
    Up2Args a;
    a.in = in; a.w = w; a.bias = bias; a.out = out;
    a.K = K; a.N = N; a.Dc = Dc; a.Vc = Vc;
    a.ntiles = (long long)B * Vc / 128;
    a.abytes = (unsigned)K / 8u * 2048u;
    a.wbytes = (unsigned)K * 16u * (unsigned)N;  // 8 N rows x K x 2 bytes
    const unsigned ncols = 8u * (unsigned)N;
    a.nsplit = ncols > 256u ? 2u : 1u;
    a.ncols_split = ncols / a.nsplit;
    a.tmem_cols = pow2_at_least(ncols);
    a.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((a.ncols_split >> 3) << 17) | ((128u >> 4) << 24);
    a.err = err;
    // at most as many CTAs per SM as their TMEM allocations fit: size the
    // shared-memory request so that no allocation has to wait
    const unsigned need = ALIGN_SLACK + UP_HDR + a.abytes + a.wbytes;
    const unsigned per_sm = 512u / a.tmem_cols;
    unsigned smem = TC_SMEM_SM / per_sm - 1024u;
    if (smem > TC_SMEM_MAX) smem = TC_SMEM_MAX;
    if (smem < need) smem = need;
    if (a.ntiles < 1) return 1;
    counted(k_up2_tc)<<<(unsigned)a.ntiles, 128, smem, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

// [taps][Npad][Kpad] (K innermost) -> [taps][Kpad / 8][Npad][8]
__global__ void k_pack_w_tc(const bf16 *__restrict__ src, int taps, int Npad, int Kpad, bf16 *__restrict__ dst)
{
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tot = (long long)taps * Npad * Kpad;
    if (e >= tot) return;
    int j = (int)(e & 7);
    long long q = e >> 3;
    int n = (int)(q % Npad);
    q /= Npad;
    int kc = (int)(q % (Kpad / 8));
    int t = (int)(q / (Kpad / 8));
    dst[e] = src[((long long)t * Npad + n) * Kpad + 8 * kc + j];
}

// [27][Npad][Kpad] -> [9 (ty, tx)][Kpad / 8][3 Npad (z-taps 2, 1, 0)][8]
__global__ void k_pack_w_tc_dzn(const bf16 *__restrict__ src, int Npad, int Kpad, bf16 *__restrict__ dst)
{
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int n3n = 3 * Npad;
    long long tot = 27LL * Npad * Kpad;
    if (e >= tot) return;
    int j = (int)(e & 7);
    long long q = e >> 3;
    int n3 = (int)(q % n3n);
    q /= n3n;
    int kc = (int)(q % (Kpad / 8));
    int yx = (int)(q / (Kpad / 8));
    int tz = 2 - n3 / Npad, n = n3 % Npad;
    int tap = 9 * tz + yx;
    dst[e] = src[((long long)tap * Npad + n) * Kpad + 8 * kc + j];
}

int pack_w_tc(const bf16 *src, int taps, int Npad, int Kpad, bf16 *dst, cudaStream_t s)
{
    if (taps == 27 && conv3_tc_dzn(Npad, Kpad)) {
        long long tot = 27LL * Npad * Kpad;
        counted(k_pack_w_tc_dzn)<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(src, Npad, Kpad, dst);
        return cudaGetLastError() == cudaSuccess ? 0 : -1;
    }
    long long tot = (long long)taps * Npad * Kpad;
    counted(k_pack_w_tc)<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(src, taps, Npad, Kpad, dst);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}


int wgrad3_tc(const bf16 *x1, int C1, const bf16 *x2, int C2, const bf16 *g, int Cg, int N, int Cw, float *dw, int B,
              int D, int *err, cudaStream_t s)
{
    const int C = C1 + C2;
    if (!(C == 16 || C == 32 || C == 64 || C == 128) || (C1 & 7) || N < 16 || N > 128 || (N & 15) || Cg < N ||
        (Cg & 7) || Cw > C || B < 1 || D < 1)
        return 0;
    if ((reinterpret_cast<uintptr_t>(x1) & 15) || (C2 > 0 && (reinterpret_cast<uintptr_t>(x2) & 15)) ||
        (reinterpret_cast<uintptr_t>(g) & 15))
        return 0;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, []() {
        attr_err = cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM_MAX);
    });
    if (attr_err != cudaSuccess) return -1;
    WgTcArgs a;
    a.x1 = x1; a.x2 = C2 > 0 ? x2 : x1; a.C1 = C1; a.C = C;
    a.g = g; a.Cg = Cg; a.N = N; a.Cw = Cw; a.dw = dw; a.B = B; a.D = D;
    a.ntap = 128 / C;
    const int ntg = (27 + a.ntap - 1) / a.ntap;
    a.V = (long long)B * D * D * D;
    const long long target = std::max(1LL, 4LL * device_sms() / ntg);
    long long chunk = (a.V + target - 1) / target;
    chunk = std::max<long long>(WG_VS, (chunk + WG_VS - 1) / WG_VS * WG_VS);
    a.chunk = chunk;
    a.nchunk = (int)((a.V + chunk - 1) / chunk);
    a.abytes = 128u * WG_VS * 2u;
    a.bbytes = (unsigned)N * WG_VS * 2u;
    a.tmem_cols = pow2_at_least((unsigned)N);
    a.idesc = (1u << 4) | (1u << 7) | (1u << 10) | (((unsigned)N >> 3) << 17) | ((128u >> 4) << 24);
    a.err = err;
    // at most as many CTAs per SM as their TMEM allocations fit
    const unsigned need = ALIGN_SLACK + WG_HDR + 2u * (a.abytes + a.bbytes);
    const unsigned per_sm = 512u / a.tmem_cols;
    unsigned smem = TC_SMEM_SM / per_sm - 1024u;
    if (smem > TC_SMEM_MAX) smem = TC_SMEM_MAX;
    if (smem < need) smem = need;
    if (smem > TC_SMEM_MAX) return 0;
    counted(k_wgrad_tc)<<<dim3((unsigned)a.nchunk, (unsigned)ntg), 128, smem, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace gnb
