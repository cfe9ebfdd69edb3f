// sort.cu -- root box, Morton keys and the space-filling-curve sort
// (tree construction, Sec. 3.4 and 5.2.2 of Hirashima et al., SC'25).
//
// Root box: lo_k = min x_k, ext = max_k(max x_k - lo_k), L = 2^ceil(log2 ext)
// (L = 1 when ext = 0), unit = L / 2^21.  Cell c_k = min(floor((x_k - lo_k) *
// 2^21 / L), 2^21 - 1) with the FP64-rounded difference; the key interleaves bit b
// of c_x, c_y, c_z at 3b+2, 3b+1, 3b.  Particles are ordered by (key, caller
// index): a stable LSD radix sort of the keys in their current slot order by
// the top 48 bits, then the short runs that agree there put in (key, caller
// index) order (see the ties section).
#include <utility>

#include "common.cuh"
#include "morton.cuh"

namespace gnb {

// ---------------------------------------------------------------- root box
__global__ void k_mm_init(unsigned long long *mm) { minmax_init(mm, threadIdx.x); }

__global__ void k_minmax(const double *__restrict__ x, const double *__restrict__ y,
                         const double *__restrict__ z, int n, unsigned long long *mm)
{
    minmax_accumulate(x, y, z, n, mm);
}

// box = {lo_x, lo_y, lo_z, L, unit}
__global__ void k_box_finalize(const unsigned long long *mm, double *box, int *status)
{
    if (threadIdx.x != 0) return;
    if (box_from_minmax(mm, box)) atomicOr(status, ST_BAD_INPUT);
}

int root_box(gnb_ctx *c)
{
    int n = (int)c->n;
    gnb::counted(k_mm_init)<<<1, 32, 0, c->s>>>(c->mm_d);
    int blocks = (n + 255) / 256;
    if (blocks > 1216) blocks = 1216;
    gnb::counted(k_minmax)<<<blocks, 256, 0, c->s>>>(c->P[c->cur].x, c->P[c->cur].y, c->P[c->cur].z, n, c->mm_d);
    gnb::counted(k_box_finalize)<<<1, 32, 0, c->s>>>(c->mm_d, c->box_d, c->status_d);
    GNB_LAUNCH_CHECK(c, "root box");
    return GNB_OK;
}

// ---------------------------------------------------------------- Morton
// Keys scattered to caller order, for the whole-key sort that a long run of
// equal 48-bit prefixes needs (see morton_and_sort).
__global__ void k_morton(PArr p, int n, const double *__restrict__ box, uint64_t *__restrict__ keyo,
                         int *__restrict__ valo, int *__restrict__ slot_of_orig)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int lexp = box_lexp(box[3]);
    const uint64_t k = morton_key(grid_cell(p.x[i], box[0], lexp), grid_cell(p.y[i], box[1], lexp),
                                  grid_cell(p.z[i], box[2], lexp));
    int o = p.orig[i];
    keyo[o] = k;
    valo[o] = o;
    slot_of_orig[o] = i;
}

// Key of every slot, paired with the slot itself for a sort in slot order
// (ties are put into caller order afterwards, see k_tie_fix), and the FP32
// remainder of each coordinate within its grid cell (res: three arrays of n,
// slot order) for the permutation.
__global__ void k_keys(const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z, int n,
                       const double *__restrict__ box, uint64_t *__restrict__ key, int *__restrict__ val,
                       float *__restrict__ res)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int lexp = box_lexp(box[3]);
    float r0, r1, r2;
    const int c0 = grid_cell(x[i], box[0], lexp, &r0);
    const int c1 = grid_cell(y[i], box[1], lexp, &r1);
    const int c2 = grid_cell(z[i], box[2], lexp, &r2);
    key[i] = morton_key(c0, c1, c2);
    val[i] = i;
    res[i] = r0;
    res[(size_t)n + i] = r1;
    res[2 * (size_t)n + i] = r2;
}

// ---------------------------------------------------------------- ties
// The slot-order sort runs over the top 48 key bits only (levels 1 to 16),
// stably, so pairs whose keys agree there are left in old-slot order; the
// order wanted is (key, caller index).  Such runs are particles in the same
// level-16 cell (a 2^-16 part of the box side), a few at most in any real
// set: one thread per run puts it in order by insertion sort, for runs of at
// most TIE_MAX entries.  st[0] = 1 when some run exists, st[1] = the longest
// (capped at TIE_MAX + 1); a longer run is left to the caller-order sort.
#define TIE_MAX 4096
#define TIE_SHIFT 16  // key bits below the sorted ones
#define TIE_FIRST_DIGIT (TIE_SHIFT / 8)

__device__ __forceinline__ bool tie(uint64_t a, uint64_t b) { return (a >> TIE_SHIFT) == (b >> TIE_SHIFT); }

__global__ void k_tie_detect(const uint64_t *__restrict__ k, int n, int *__restrict__ st)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i + 1 >= n || !tie(k[i], k[i + 1])) return;
    if (i > 0 && tie(k[i - 1], k[i])) return;  // not the run's start
    int e = i + 1;
    while (e < n && e - i <= TIE_MAX && tie(k[e], k[i])) e++;
    atomicOr(&st[0], 1);
    atomicMax(&st[1], e - i);
}

__global__ void k_tie_fix(uint64_t *__restrict__ k, int n, int *__restrict__ val, const int *__restrict__ orig)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i + 1 >= n || !tie(k[i], k[i + 1])) return;
    if (i > 0 && tie(k[i - 1], k[i])) return;
    int e = i + 1;
    while (e < n && tie(k[e], k[i])) e++;
    for (int a = i + 1; a < e; a++) {  // insertion sort of the pairs [i, e) by (key, orig[val])
        const uint64_t kv = k[a];
        const int v = val[a], ov = orig[v];
        int b = a - 1;
        while (b >= i && (k[b] > kv || (k[b] == kv && orig[val[b]] > ov))) {
            k[b + 1] = k[b];
            val[b + 1] = val[b];
            b--;
        }
        k[b + 1] = kv;
        val[b + 1] = v;
    }
}

// ---------------------------------------------------------------- radix sort
// Stable LSD radix sort of (64-bit key, 32-bit value), 8 bits per pass.
// Tiles of RS_TILE keys; per pass: digit histogram per tile, per-digit scan
// over tiles, stable scatter with per-warp match ranks.
#define RS_THREADS 256
#define RS_ITEMS 16
#define RS_TILE (RS_THREADS * RS_ITEMS)

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint64_t *__restrict__ k, int n, int shift,
                                                       int *__restrict__ counts, int ntiles,
                                                       int *__restrict__ total)
{
    __shared__ int h[256];
    int t = threadIdx.x, tile = blockIdx.x;
    h[t] = 0;
    __syncthreads();
    int base = tile * RS_TILE;
#pragma unroll
    for (int r = 0; r < RS_ITEMS; r++) {
        int i = base + r * RS_THREADS + t;
        if (i < n) atomicAdd(&h[(int)((k[i] >> shift) & 255u)], 1);
    }
    __syncthreads();
    int v = h[t];
    counts[t * ntiles + tile] = v;
    if (v) atomicAdd(&total[t], v);
}

// One block per digit: offs[d][tile] = base(d) + sum_{t' < tile} counts[d][t'].
__global__ void __launch_bounds__(1024) k_rs_scan(int *__restrict__ counts, int ntiles,
                                                  const int *__restrict__ total)
{
    __shared__ int wsum[32];
    __shared__ int s_base, s_carry;
    int d = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t < 32) {
        int acc = 0;
        for (int e = lane; e < d; e += 32) acc += total[e];
        acc = warp_sum(acc);
        if (lane == 0) { s_base = acc; s_carry = 0; }
    }
    __syncthreads();
    int *row = counts + (size_t)d * ntiles;
    for (int b0 = 0; b0 < ntiles; b0 += 1024) {
        int i = b0 + t;
        int v = i < ntiles ? row[i] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            int s = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            wsum[lane] = s;
        }
        __syncthreads();
        int excl = x - v + (w > 0 ? wsum[w - 1] : 0);
        if (i < ntiles) row[i] = s_base + s_carry + excl;
        __syncthreads();
        if (t == 0) s_carry += wsum[31];
        __syncthreads();
    }
}

// Scatter of one tile: the tile's pairs are first sorted by digit in shared
// memory, stably, then written out in that order, so consecutive threads
// write consecutive addresses of each digit's run (about RS_TILE / 256 pairs
// per digit) instead of one scattered 8-byte store each.  Each warp ranks its
// own contiguous RS_ITEMS * 32 pairs of the tile (rounds of 32 in order,
// lanes in order within a round) against per-warp digit counters, with warp
// synchronisation only; one block-wide step then turns the counters into each
// warp's offset within the digit's run of the tile.
struct RsSmem {
    uint64_t k[RS_TILE];
    int v[RS_TILE];
    int wc[RS_THREADS / 32][256];  // per-warp digit counts, then each warp's offset in the digit's run
    int lstart[256];               // first local position of each digit
    int goff[256];                 // global position of each digit's first pair of this tile
    int ws[RS_THREADS / 32];
};

__global__ void __launch_bounds__(RS_THREADS, 3) k_rs_scatter(const uint64_t *__restrict__ kin,
                                                          const int *__restrict__ vin,
                                                          uint64_t *__restrict__ kout,
                                                          int *__restrict__ vout, int n, int shift,
                                                          const int *__restrict__ offs, int ntiles)
{
    extern __shared__ __align__(16) unsigned char rs_raw[];
    RsSmem &S = *reinterpret_cast<RsSmem *>(rs_raw);
    const int t = threadIdx.x, tile = blockIdx.x, w = t >> 5, lane = t & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int base = tile * RS_TILE;
    const int cnt = min(RS_TILE, n - base);
#pragma unroll
    for (int q = 0; q < RS_THREADS / 32; q++) S.wc[q][t] = 0;
    S.goff[t] = offs[t * ntiles + tile];
    __syncthreads();
    uint64_t key[RS_ITEMS];
    int val[RS_ITEMS], lr[RS_ITEMS];
#pragma unroll
    for (int r = 0; r < RS_ITEMS; r++) {
        const int i = w * (RS_ITEMS * 32) + r * 32 + lane;
        const bool valid = i < cnt;
        key[r] = valid ? kin[base + i] : 0ull;
        val[r] = valid ? vin[base + i] : 0;
        const int d = valid ? (int)((key[r] >> shift) & 255u) : 256;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int leader = __ffs(peers) - 1;
        int old = 0;
        if (valid && lane == leader) {
            old = S.wc[w][d];
            S.wc[w][d] = old + __popc(peers);
        }
        old = __shfl_sync(0xffffffffu, old, leader);
        lr[r] = old + __popc(peers & lt);
        __syncwarp();
    }
    __syncthreads();
    {   // digit t: offsets of the warps within the digit's run, then the
        // exclusive scan of the tile histogram over the 256 digits
        int run = 0;
#pragma unroll
        for (int q = 0; q < RS_THREADS / 32; q++) {
            const int c = S.wc[q][t];
            S.wc[q][t] = run;
            run += c;
        }
        int x = run;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) S.ws[w] = x;
        __syncthreads();
        int pre = 0;
        for (int q = 0; q < w; q++) pre += S.ws[q];
        S.lstart[t] = pre + x - run;
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < RS_ITEMS; r++) {
        const int i = w * (RS_ITEMS * 32) + r * 32 + lane;
        if (i < cnt) {
            const int d = (int)((key[r] >> shift) & 255u);
            const int lp = S.lstart[d] + S.wc[w][d] + lr[r];
            S.k[lp] = key[r];
            S.v[lp] = val[r];
        }
    }
    __syncthreads();
    for (int pos = t; pos < cnt; pos += RS_THREADS) {
        const uint64_t k = S.k[pos];
        const int d = (int)((k >> shift) & 255u);
        const int dst = S.goff[d] + pos - S.lstart[d];
        kout[dst] = k;
        vout[dst] = S.v[pos];
    }
}

// The scatter's tile (about 59 KB) needs the opt-in to more than 48 KB of
// dynamic shared memory.
static int rs_scatter_attr(gnb_ctx *c)
{
    cudaError_t e = cudaFuncSetAttribute(k_rs_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(RsSmem));
    return e == cudaSuccess ? GNB_OK : cuda_check(c, e, "radix sort shared memory attribute");
}

// Stable sort of n (64-bit key, 32-bit value) pairs held in (k0, v0) by the
// key bits from 8 first_digit up (first_digit even), with (k1, v1) as the
// ping-pong buffers; the sorted pairs end in (k0, v0).
int radix_sort_pairs(gnb_ctx *c, uint64_t *k0, int *v0, uint64_t *k1, int *v1, int n, int first_digit)
{
    int ntiles = (n + RS_TILE - 1) / RS_TILE;
    GNB_TRY(rs_scatter_attr(c));
    uint64_t *kin = k0, *kout = k1;
    int *vin = v0, *vout = v1;
    for (int pass = first_digit; pass < 8; pass++) {
        int shift = 8 * pass;
        cudaMemsetAsync(c->rs_total, 0, 256 * sizeof(int), c->s);
        gnb::counted(k_rs_hist)<<<ntiles, RS_THREADS, 0, c->s>>>(kin, n, shift, c->rs_counts, ntiles, c->rs_total);
        gnb::counted(k_rs_scan)<<<256, 1024, 0, c->s>>>(c->rs_counts, ntiles, c->rs_total);
        gnb::counted(k_rs_scatter)<<<ntiles, RS_THREADS, sizeof(RsSmem), c->s>>>(kin, vin, kout, vout, n, shift,
                                                                                  c->rs_counts,
                                                                    ntiles);
        uint64_t *tk = kin; kin = kout; kout = tk;
        int *tv = vin; vin = vout; vout = tv;
    }
    GNB_LAUNCH_CHECK(c, "radix sort");
    return GNB_OK;
}

// ---------------------------------------------------------------- permute
// New slot i takes old slot src[i] = slot_of_orig[sorted caller index].
__global__ void k_src(const int *__restrict__ sval, const int *__restrict__ slot_of_orig,
                      int *__restrict__ src, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) src[i] = slot_of_orig[sval[i]];
}

// New slot i takes old slot src[i]; its grid cell comes from its sorted key
// and its remainder within the cell from the key pass (res, old-slot order).
__global__ void k_permute(PArr a, PArr b, const int *__restrict__ src, int n, const uint64_t *__restrict__ skey,
                          const float *__restrict__ res)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int s = src[i];
    b.x[i] = a.x[s]; b.y[i] = a.y[s]; b.z[i] = a.z[s]; b.h2[i] = a.h2[s]; b.id[i] = a.id[s];
    b.vx[i] = a.vx[s]; b.vy[i] = a.vy[s]; b.vz[i] = a.vz[s];
    b.m[i] = a.m[s]; b.eps[i] = a.eps[s]; b.u[i] = a.u[s];
    b.vpx[i] = a.vpx[s]; b.vpy[i] = a.vpy[s]; b.vpz[i] = a.vpz[s]; b.up[i] = a.up[s];
    b.orig[i] = a.orig[s]; b.grank[i] = a.grank[s];
    b.type[i] = a.type[s];
    const uint64_t k = skey[i];
    b.cx[i] = compact3(k >> 2);
    b.cy[i] = compact3(k >> 1);
    b.cz[i] = compact3(k);
    b.rx[i] = res[s];
    b.ry[i] = res[(size_t)n + s];
    b.rz[i] = res[2 * (size_t)n + s];
}

// The first sort after an upload starts from the caller's order, so its
// gather sources are spread over whole arrays: one pass per array keeps that
// array (at most 8 bytes a particle) in L2 while it is gathered, instead of
// one pass whose 22 sources together are far larger than L2 (on the 2^24
// disk the single pass took 7.1 ms against 0.73 ms for the near-sorted
// permutations of later steps).
template <class T>
__global__ void k_gather1(const T *__restrict__ a, T *__restrict__ b, const int *__restrict__ src, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[src[i]];
}

__global__ void k_cells_of_key(const uint64_t *__restrict__ skey, int n, int *__restrict__ cx, int *__restrict__ cy,
                               int *__restrict__ cz)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t k = skey[i];
    cx[i] = compact3(k >> 2);
    cy[i] = compact3(k >> 1);
    cz[i] = compact3(k);
}

template <class T>
static void gather1(gnb_ctx *c, const T *a, T *b, const int *src, int n)
{
    gnb::counted(k_gather1<T>)<<<(n + 255) / 256, 256, 0, c->s>>>(a, b, src, n);
}

static int permute_per_array(gnb_ctx *c, const PArr &a, PArr &b, const int *src, int n)
{
    for (auto q : {std::make_pair(a.x, b.x), std::make_pair(a.y, b.y), std::make_pair(a.z, b.z),
                   std::make_pair(a.h2, b.h2)})
        gather1<double>(c, q.first, q.second, src, n);
    gather1<int64_t>(c, a.id, b.id, src, n);
    for (auto q : {std::make_pair(a.vx, b.vx), std::make_pair(a.vy, b.vy), std::make_pair(a.vz, b.vz),
                   std::make_pair(a.m, b.m), std::make_pair(a.eps, b.eps), std::make_pair(a.u, b.u),
                   std::make_pair(a.vpx, b.vpx), std::make_pair(a.vpy, b.vpy), std::make_pair(a.vpz, b.vpz),
                   std::make_pair(a.up, b.up)})
        gather1<float>(c, q.first, q.second, src, n);
    const float *res = c->kres;
    gather1<float>(c, res, b.rx, src, n);
    gather1<float>(c, res + (size_t)n, b.ry, src, n);
    gather1<float>(c, res + 2 * (size_t)n, b.rz, src, n);
    gather1<int>(c, a.orig, b.orig, src, n);
    gather1<int>(c, a.grank, b.grank, src, n);
    gather1<uint8_t>(c, a.type, b.type, src, n);
    gnb::counted(k_cells_of_key)<<<(n + 255) / 256, 256, 0, c->s>>>(c->skey, n, b.cx, b.cy, b.cz);
    GNB_LAUNCH_CHECK(c, "permute per array");
    return GNB_OK;
}

int morton_and_sort(gnb_ctx *c)
{
    int n = (int)c->n;
    GNB_TRY(root_box(c));
    int nb = (n + 255) / 256;
    PArr &a = c->P[c->cur];
    // keys in slot order (the particles are near their previous Morton
    // order), stable sort by the top 48 bits, then runs into (key, caller
    // index) order
    gnb::counted(k_keys)<<<nb, 256, 0, c->s>>>(a.x, a.y, a.z, n, c->box_d, c->skey, c->sval, c->kres);
    GNB_LAUNCH_CHECK(c, "keys");
    GNB_TRY(radix_sort_pairs(c, c->skey, c->sval, c->skey2, c->sval2, n, TIE_FIRST_DIGIT));
    cudaMemsetAsync(c->work_d + 2, 0, 2 * sizeof(int), c->s);
    gnb::counted(k_tie_detect)<<<nb, 256, 0, c->s>>>(c->skey, n, c->work_d + 2);
    GNB_LAUNCH_CHECK(c, "tie detect");
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(c->pinned_i + 60, c->work_d + 2, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                                          c->s), "tie flag"));
    GNB_TRY(cuda_check(c, cudaStreamSynchronize(c->s), "tie flag sync"));
    const int *src = c->sval;  // the old slot of each sorted particle
    if (c->pinned_i[60] && c->pinned_i[61] <= TIE_MAX) {
        gnb::counted(k_tie_fix)<<<nb, 256, 0, c->s>>>(c->skey, n, c->sval, a.orig);
        GNB_LAUNCH_CHECK(c, "tie fix");
    } else if (c->pinned_i[60]) {
        // a run of more than TIE_MAX: sort by the whole key in caller order
        // (keys scattered to the caller index, stable sort, slot map)
        gnb::counted(k_morton)<<<nb, 256, 0, c->s>>>(a, n, c->box_d, c->skey, c->sval, c->slot_of_orig);
        GNB_LAUNCH_CHECK(c, "morton");
        GNB_TRY(radix_sort_pairs(c, c->skey, c->sval, c->skey2, c->sval2, n, 0));
        gnb::counted(k_src)<<<nb, 256, 0, c->s>>>(c->sval, c->slot_of_orig, c->src, n);
        src = c->src;
    }
    if (src != c->src)
        GNB_TRY(cuda_check(c, cudaMemcpyAsync(c->src, src, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, c->s),
                           "slot map copy"));
    PArr &b = c->P[1 - c->cur];
    if (c->slots_caller) {
        GNB_TRY(permute_per_array(c, a, b, c->src, n));
        c->slots_caller = false;
    } else {
        gnb::counted(k_permute)<<<nb, 256, 0, c->s>>>(a, b, c->src, n, c->skey, c->kres);
        GNB_LAUNCH_CHECK(c, "permute");
    }
    c->cur = 1 - c->cur;
    if (c->hier_on) GNB_TRY(hier_permute(c));  // per-particle step state follows the particles
    return GNB_OK;
}

}  // namespace gnb
