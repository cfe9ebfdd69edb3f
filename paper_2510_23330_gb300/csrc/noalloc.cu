// noalloc.cu -- Morton keys and space-filling-curve order with no device
// allocation (gnb_morton_order_noalloc in galnb.h).
//
// Some callers cannot allocate device memory: an application whose device
// memory is owned by another allocator (a framework's caching pool or a
// fixed arena), or a latency-sensitive loop in which cudaMalloc/cudaFree
// would synchronise the device or could fail under memory pressure.  For
// them this file computes the same keys and order as the context path (root
// box, keys, stable LSD radix sort by (key, caller index)) with all scratch
// in one file-scope static device array of fixed size.  The array exists on
// every GPU that loads the library, until the process exits.  Host code must
// not pass the array's name to a kernel (on the host it is only a stand-in):
// the device address is looked up once per device with cudaGetSymbolAddress
// and passed to the kernels.
#include <mutex>

#include "common.cuh"
#include "morton.cuh"

namespace gnb {
namespace {

constexpr int NA_MAX = GNB_NOALLOC_MAX_N;
constexpr int NA_THREADS = 256;
constexpr int NA_ITEMS = 8;
constexpr int NA_TILE = NA_THREADS * NA_ITEMS;
constexpr int NA_TILES = (NA_MAX + NA_TILE - 1) / NA_TILE;

// scratch layout (byte offsets, each region 256-byte aligned)
constexpr size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t OFF_KEYA = 0;
constexpr size_t OFF_KEYB = OFF_KEYA + al256(sizeof(uint64_t) * NA_MAX);
constexpr size_t OFF_VALA = OFF_KEYB + al256(sizeof(uint64_t) * NA_MAX);
constexpr size_t OFF_VALB = OFF_VALA + al256(sizeof(int) * NA_MAX);
constexpr size_t OFF_CNT = OFF_VALB + al256(sizeof(int) * NA_MAX);
constexpr size_t OFF_TOT = OFF_CNT + al256(sizeof(int) * 256 * NA_TILES);
constexpr size_t OFF_MM = OFF_TOT + al256(sizeof(int) * 256);
constexpr size_t OFF_BOX = OFF_MM + al256(sizeof(unsigned long long) * 8);
constexpr size_t OFF_FLAG = OFF_BOX + al256(sizeof(double) * 8);
constexpr size_t SCRATCH_BYTES = OFF_FLAG + al256(sizeof(int) * 4);

static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

// Clears what must start at zero (or at the min/max sentinels) every call.
__global__ void k_na_init(unsigned char *scr)
{
    minmax_init((unsigned long long *)(scr + OFF_MM), threadIdx.x);
    if (threadIdx.x == 0) ((int *)(scr + OFF_FLAG))[0] = 0;
}

// The root box and the keys come from the same device functions as the
// context path (morton.cuh), so both paths give the same bits.
__global__ void k_na_minmax(const double *__restrict__ x, const double *__restrict__ y,
                            const double *__restrict__ z, int n, unsigned char *scr)
{
    minmax_accumulate(x, y, z, n, (unsigned long long *)(scr + OFF_MM));
}

// box = {lo x, lo y, lo z, L, unit}: lo = minimum, L = power of two >= extent
__global__ void k_na_box(unsigned char *scr)
{
    if (threadIdx.x != 0) return;
    if (box_from_minmax((const unsigned long long *)(scr + OFF_MM), (double *)(scr + OFF_BOX)))
        ((int *)(scr + OFF_FLAG))[0] = 1;
}

__global__ void k_na_keys(const double *__restrict__ x, const double *__restrict__ y,
                          const double *__restrict__ z, int n, const unsigned char *scr,
                          uint64_t *__restrict__ keys)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *box = (const double *)(scr + OFF_BOX);
    const int lexp = box_lexp(box[3]);
    keys[i] = morton_key(grid_cell(x[i], box[0], lexp), grid_cell(y[i], box[1], lexp), grid_cell(z[i], box[2], lexp));
}

__global__ void __launch_bounds__(NA_THREADS) k_na_hist(const uint64_t *__restrict__ k, int n, int shift,
                                                       unsigned char *scr, int ntiles)
{
    int *counts = (int *)(scr + OFF_CNT);
    int *total = (int *)(scr + OFF_TOT);
    __shared__ int h[256];
    int t = threadIdx.x, tile = blockIdx.x;
    h[t] = 0;
    __syncthreads();
    int base = tile * NA_TILE;
#pragma unroll
    for (int r = 0; r < NA_ITEMS; r++) {
        int i = base + r * NA_THREADS + t;
        if (i < n) atomicAdd(&h[(int)((k[i] >> shift) & 255u)], 1);
    }
    __syncthreads();
    int v = h[t];
    counts[t * ntiles + tile] = v;
    if (v) atomicAdd(&total[t], v);
}

// one block per digit: exclusive offsets over (digit, tile)
__global__ void __launch_bounds__(NA_TILES) k_na_scan(unsigned char *scr, int ntiles)
{
    int *counts = (int *)(scr + OFF_CNT);
    const int *total = (const int *)(scr + OFF_TOT);
    __shared__ int ws[NA_TILES / 32];
    __shared__ int s_base;
    int d = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t < 32) {
        int acc = 0;
        for (int e = lane; e < d; e += 32) acc += total[e];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) s_base = acc;
    }
    int v = t < ntiles ? counts[d * ntiles + t] : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    int pre = 0;
    for (int q = 0; q < w; q++) pre += ws[q];
    if (t < ntiles) counts[d * ntiles + t] = s_base + pre + x - v;
}

// stable scatter; vin == nullptr means the values are the indices 0..n-1
__global__ void __launch_bounds__(NA_THREADS) k_na_scatter(const uint64_t *__restrict__ kin,
                                                          const int *__restrict__ vin, uint64_t *__restrict__ kout,
                                                          int *__restrict__ vout, int n, int shift,
                                                          const unsigned char *scr, int ntiles)
{
    const int *offs = (const int *)(scr + OFF_CNT);
    __shared__ int s_w[8][256];
    __shared__ int s_run[256];
    __shared__ int s_off[256];
    int t = threadIdx.x, tile = blockIdx.x, w = t >> 5, lane = t & 31;
    s_run[t] = 0;
    s_off[t] = offs[t * ntiles + tile];
    unsigned lt = (1u << lane) - 1u;
    int base = tile * NA_TILE;
    for (int r = 0; r < NA_ITEMS; r++) {
#pragma unroll
        for (int q = 0; q < 8; q++) s_w[q][t] = 0;
        __syncthreads();
        int i = base + r * NA_THREADS + t;
        bool valid = i < n;
        uint64_t key = valid ? kin[i] : 0ull;
        int d = valid ? (int)((key >> shift) & 255u) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & lt);
        if (valid && rank == 0) s_w[w][d] = __popc(peers);
        __syncthreads();
        {
            int run = s_run[t];
#pragma unroll
            for (int q = 0; q < 8; q++) {
                int cnt = s_w[q][t];
                s_w[q][t] = run;
                run += cnt;
            }
            s_run[t] = run;
        }
        __syncthreads();
        if (valid) {
            int dst = s_off[d] + s_w[w][d] + rank;
            kout[dst] = key;
            vout[dst] = vin ? vin[i] : i;
        }
        __syncthreads();
    }
}

__global__ void k_na_order(const int *__restrict__ v, int n, int64_t *__restrict__ order)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) order[i] = v[i];
}

std::mutex g_na_mu;
void *g_na_ptr[64] = {nullptr};

// Device address of the scratch array on the current device (looked up on
// the first call on each device).
int na_scratch(unsigned char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GNB_ECUDA;
    }
    if (dev < 0 || dev >= 64) return GNB_EINVAL;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return GNB_ECUDA;
        }
        g_na_ptr[dev] = p;
    }
    *out = (unsigned char *)g_na_ptr[dev];
    return GNB_OK;
}

}  // namespace
}  // namespace gnb

extern "C" int gnb_morton_order_noalloc(int64_t n, const double *x, const double *y, const double *z,
                                        uint64_t *keys, int64_t *order, void *stream)
{
    using namespace gnb;
    if (n < 1 || n > NA_MAX) return GNB_EINVAL;
    if (!x || !y || !z || !keys || !order) return GNB_EINVAL;
    unsigned char *scr = nullptr;
    int rc = na_scratch(&scr);
    if (rc != GNB_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    int ni = (int)n;
    int nb = (ni + 255) / 256;
    int ntiles = (ni + NA_TILE - 1) / NA_TILE;
    counted(k_na_init)<<<1, 32, 0, s>>>(scr);
    counted(k_na_minmax)<<<nb < 1216 ? nb : 1216, 256, 0, s>>>(x, y, z, ni, scr);
    counted(k_na_box)<<<1, 32, 0, s>>>(scr);
    counted(k_na_keys)<<<nb, 256, 0, s>>>(x, y, z, ni, scr, keys);
    uint64_t *ka = (uint64_t *)(scr + OFF_KEYA), *kb = (uint64_t *)(scr + OFF_KEYB);
    int *va = (int *)(scr + OFF_VALA), *vb = (int *)(scr + OFF_VALB);
    const uint64_t *kin = keys;
    const int *vin = nullptr;
    for (int pass = 0; pass < 8; pass++) {
        uint64_t *kout = (pass & 1) ? kb : ka;
        int *vout = (pass & 1) ? vb : va;
        cudaMemsetAsync(scr + OFF_TOT, 0, sizeof(int) * 256, s);
        counted(k_na_hist)<<<ntiles, NA_THREADS, 0, s>>>(kin, ni, 8 * pass, scr, ntiles);
        counted(k_na_scan)<<<256, NA_TILES, 0, s>>>(scr, ntiles);
        counted(k_na_scatter)<<<ntiles, NA_THREADS, 0, s>>>(kin, vin, kout, vout, ni, 8 * pass, scr, ntiles);
        kin = kout;
        vin = vout;
    }
    counted(k_na_order)<<<nb, 256, 0, s>>>(vin, ni, order);
    if (cudaGetLastError() != cudaSuccess) return GNB_ECUDA;
    int flag = 0;
    if (cudaMemcpyAsync(&flag, scr + OFF_FLAG, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return GNB_ECUDA;
    }
    return flag ? GNB_EINVAL : GNB_OK;
}
