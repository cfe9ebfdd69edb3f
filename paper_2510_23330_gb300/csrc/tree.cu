// tree.cu -- octree over Morton-sorted particles, cell moments and groups
// (Barnes-Hut treecode, Sec. 1 and 3.4; groups sharing one interaction list,
// Sec. 5.2.2 and 5.2.4 of Hirashima et al., SC'25).
//
// A level-l cell holds the particles sharing the top 3l key bits.  A cell is
// split when it holds more than n_leaf particles and l < 21; its non-empty
// children are stored in Morton order.  The node array is the breadth-first
// list (level by level, Morton order within a level), built in a fixed
// number of passes over the sorted keys whatever the depth (see the build
// section); level bounds live in t.lvl: level l is [lvl[l], lvl[l+1]).
//
// Moments are FP32 about each cell's integer corner: M, centre of mass
// offset, traceless quadrupole Q = sum m (3 d d - d^2 I) about the centre of
// mass, and the mass-weighted mean eps^2.  Parents combine their children
// with the parallel-axis shift.
#include "common.cuh"
#include "morton.cuh"

namespace gnb {

#define TB_THREADS 256
#define TB_BLOCKS 304

// ----------------------------------------------------------------- scan
// Block b scans the contiguous chunk [b chunk, (b + 1) chunk) of the input,
// four elements a thread per round (one 16-byte load; the inputs are
// allocation bases, so 16-byte aligned), with chunk a multiple of the
// TB_THREADS * 4 elements of a round.
__device__ __forceinline__ int scan_chunk(int n, int G)
{
    const int per = (n + G - 1) / G;
    return (per + TB_THREADS * 4 - 1) / (TB_THREADS * 4) * (TB_THREADS * 4);
}

__device__ __forceinline__ int4 load4(const int *__restrict__ in, int i0, int end)
{
    if (i0 + 3 < end) return *reinterpret_cast<const int4 *>(in + i0);
    return make_int4(i0 < end ? in[i0] : 0, i0 + 1 < end ? in[i0 + 1] : 0, i0 + 2 < end ? in[i0 + 2] : 0, 0);
}

__global__ void k_scan_partial(const int *__restrict__ in, const int *__restrict__ n_d, int *partial)
{
    __shared__ int ws[32];
    int n = *n_d, G = gridDim.x;
    int chunk = scan_chunk(n, G);
    int beg = min(n, blockIdx.x * chunk), end = min(n, beg + chunk);
    int s = 0;
    for (int i0 = beg + 4 * threadIdx.x; i0 < end; i0 += 4 * blockDim.x) {
        const int4 v = load4(in, i0, end);
        s += v.x + v.y + v.z + v.w;
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        int v = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0;
        v = warp_sum(v);
        if (threadIdx.x == 0) partial[blockIdx.x] = v;
    }
}

// Exclusive scan of G <= 1024 partials into poff; poff[G] = total.
__global__ void k_scan_partials(const int *__restrict__ partial, int *poff, int G, int *total_d)
{
    __shared__ int ws[32];
    int t = threadIdx.x, lane = t & 31, w = t >> 5;
    int v = t < G ? partial[t] : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = ws[lane];
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        ws[lane] = s;
    }
    __syncthreads();
    int excl = x - v + (w > 0 ? ws[w - 1] : 0);
    if (t < G) poff[t] = excl;
    if (t == 1023) {
        poff[G] = ws[31];
        if (total_d) *total_d = ws[31];
    }
}

// Block-level exclusive scan helper: returns the exclusive prefix of v over
// the block and writes the block total to *tot.
__device__ __forceinline__ int block_excl_scan(int v, int *ws, int *tot)
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

__global__ void k_scan_apply(const int *__restrict__ in, int *__restrict__ out, const int *__restrict__ n_d,
                             const int *__restrict__ poff)
{
    __shared__ int ws[32];
    int n = *n_d, G = gridDim.x;
    int chunk = scan_chunk(n, G);
    int beg = min(n, blockIdx.x * chunk), end = min(n, beg + chunk);
    int carry = poff[blockIdx.x];
    for (int b0 = beg; b0 < end; b0 += 4 * blockDim.x) {
        const int i0 = b0 + 4 * threadIdx.x;
        const int4 v = load4(in, i0, end);
        int tot;
        const int e = carry + block_excl_scan(v.x + v.y + v.z + v.w, ws, &tot);
        const int4 o = make_int4(e, e + v.x, e + v.x + v.y, e + v.x + v.y + v.z);
        if (i0 + 3 < end) {
            *reinterpret_cast<int4 *>(out + i0) = o;
        } else {
            if (i0 < end) out[i0] = o.x;
            if (i0 + 1 < end) out[i0 + 1] = o.y;
            if (i0 + 2 < end) out[i0 + 2] = o.z;
        }
        carry += tot;
    }
}

// Slots of the gas particles in slot order, straight from the type bytes:
// per-block gas counts over the same chunks as the scan (16 types a thread
// per round, one 16-byte load), then each block writes its gas slots from the
// scanned counts.
#define GC_ITEMS 16
__device__ __forceinline__ int gas_chunk(int n, int G)
{
    const int per = (n + G - 1) / G;
    return (per + TB_THREADS * GC_ITEMS - 1) / (TB_THREADS * GC_ITEMS) * (TB_THREADS * GC_ITEMS);
}

// bit k set when type byte k of the 16 at i0 is gas (bytes past end: not gas)
__device__ __forceinline__ unsigned gas_mask16(const uint8_t *__restrict__ type, int i0, int end)
{
    unsigned m = 0u;
    if (i0 + GC_ITEMS <= end) {
        const uint4 v = *reinterpret_cast<const uint4 *>(type + i0);
        const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; q++)
#pragma unroll
            for (int b = 0; b < 4; b++)
                if (((w[q] >> (8 * b)) & 255u) == GNB_GAS) m |= 1u << (4 * q + b);
    } else {
        for (int k = 0; k < GC_ITEMS && i0 + k < end; k++)
            if (type[i0 + k] == GNB_GAS) m |= 1u << k;
    }
    return m;
}

__global__ void k_gas_count(const uint8_t *__restrict__ type, const int *__restrict__ n_d, int *partial)
{
    __shared__ int ws[32];
    const int n = *n_d, G = gridDim.x;
    const int chunk = gas_chunk(n, G);
    const int beg = min(n, blockIdx.x * chunk), end = min(n, beg + chunk);
    int s = 0;
    for (int i0 = beg + GC_ITEMS * threadIdx.x; i0 < end; i0 += GC_ITEMS * blockDim.x)
        s += __popc(gas_mask16(type, i0, end));
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        int v = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0;
        v = warp_sum(v);
        if (threadIdx.x == 0) partial[blockIdx.x] = v;
    }
}

__global__ void k_gas_slots(const uint8_t *__restrict__ type, const int *__restrict__ n_d,
                            const int *__restrict__ poff, int *__restrict__ gslot)
{
    __shared__ int ws[32];
    const int n = *n_d, G = gridDim.x;
    const int chunk = gas_chunk(n, G);
    const int beg = min(n, blockIdx.x * chunk), end = min(n, beg + chunk);
    int carry = poff[blockIdx.x];
    for (int b0 = beg; b0 < end; b0 += GC_ITEMS * blockDim.x) {
        const int i0 = b0 + GC_ITEMS * threadIdx.x;
        unsigned m = i0 < end ? gas_mask16(type, i0, end) : 0u;
        int tot;
        int pos = carry + block_excl_scan(__popc(m), ws, &tot);
        while (m) {
            const int k = __ffs(m) - 1;
            gslot[pos++] = i0 + k;
            m &= m - 1u;
        }
        carry += tot;
    }
}

int gas_slots(gnb_ctx *c, const uint8_t *type, const int *n_d, int *gslot)
{
    gnb::counted(k_gas_count)<<<TB_BLOCKS, TB_THREADS, 0, c->s>>>(type, n_d, c->scan_part);
    gnb::counted(k_scan_partials)<<<1, 1024, 0, c->s>>>(c->scan_part, c->scan_poff, TB_BLOCKS, nullptr);
    gnb::counted(k_gas_slots)<<<TB_BLOCKS, TB_THREADS, 0, c->s>>>(type, n_d, c->scan_poff, gslot);
    GNB_LAUNCH_CHECK(c, "gas slots");
    return GNB_OK;
}

int device_scan(gnb_ctx *c, const int *in, int *out, const int *n_d, int nmax, int *total_d)
{
    (void)nmax;
    gnb::counted(k_scan_partial)<<<TB_BLOCKS, TB_THREADS, 0, c->s>>>(in, n_d, c->scan_part);
    gnb::counted(k_scan_partials)<<<1, 1024, 0, c->s>>>(c->scan_part, c->scan_poff, TB_BLOCKS, total_d);
    gnb::counted(k_scan_apply)<<<TB_BLOCKS, TB_THREADS, 0, c->s>>>(in, out, n_d, c->scan_poff);
    GNB_LAUNCH_CHECK(c, "scan");
    return GNB_OK;
}


// ----------------------------------------------------------------- build
// The node set follows from the sorted keys alone.  Slot i starts a level-l
// cell when it shares fewer than l leading octal digits with slot i - 1; the
// cell is a node when its parent cell holds more than n_leaf particles (the
// parent is split; every ancestor then holds more too, so it exists); it is
// split when it holds more than n_leaf and l < 21.  The level-l cell that
// starts at i holds more than m particles iff slot i + m exists and shares
// l digits with i.  So slot i starts the nodes of levels a_i .. b_i, with
// a_i = (digits shared with slot i - 1) + 1 and b_i the first level whose
// cell holds at most n_leaf (or 21): three passes over the keys, whatever
// the depth -- spans and per-tile counts, one scan per level over the tiles,
// emission of the breadth-first node array (level by level, in slot order
// within a level).

#define TB_ITEMS 16
#define TB_TILE (TB_THREADS * TB_ITEMS)
#define TB_NCNT (GNB_MAXLEV + 2)  // a counter per level, then one for the groups

// leading octal digits two keys share (21 when equal; bit 63 of a key is 0)
__device__ __forceinline__ int shared_levels(uint64_t a, uint64_t b)
{
    return (__clzll((long long)(a ^ b)) - 1) / 3;
}

// The sorted keys, read through the read-only data cache.
struct KeyWin {
    const uint64_t *__restrict__ k;
    __device__ __forceinline__ uint64_t operator()(int j) const { return __ldg(k + j); }
};

// whether two keys lie in the same level-l cell (0 <= l <= 21)
__device__ __forceinline__ bool same_cell(uint64_t a, uint64_t b, int l)
{
    return ((a ^ b) >> (63 - 3 * l)) == 0;
}

// whether the level-l cell that starts at slot s holds more than m particles
__device__ __forceinline__ bool cell_gt(const KeyWin &k, int n, int s, int m, int l)
{
    return s + m < n && same_cell(k(s), k(s + m), l);
}

// whether the level-l cell holding slot i holds more than m particles: it
// does if it reaches back to slot i - m - 1; else it starts within the m
// slots before i, found by bisection
__device__ bool holder_gt(const KeyWin &k, int n, int i, int l, int m)
{
    const uint64_t ki = k(i);
    int lo = i - m - 1;
    if (lo >= 0 && same_cell(k(lo), ki, l)) return true;
    lo = max(lo + 1, 0);
    int hi = i;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (same_cell(k(mid), ki, l)) hi = mid;
        else lo = mid + 1;
    }
    return cell_gt(k, n, lo, m, l);
}

// span of slot i: bit 24 set when nodes start there, bits 0-7 the first
// level a, 8-15 the last level b, 16-23 one more than the level of the group
// starting there (0: none).  A group is the first node on its root-to-leaf
// path that holds at most n_g particles or is a leaf; at slot i that is
// level min(b, max(a, g + 1)), g = digits shared with slot i + n_g, whose
// parent holds more than n_g unless it is level a > 0, where the parent
// cell starts before i and is tested like the split.
__device__ int span_of(const KeyWin &k, int n, int i, int n_leaf, int n_g)
{
    int a = 0;
    const uint64_t ki = k(i);
    if (i > 0) {
        const int d = shared_levels(k(i - 1), ki);
        if (d >= GNB_MAXLEV || !holder_gt(k, n, i, d, n_leaf)) return 0;
        a = d + 1;
    }
    const int q = i + n_leaf < n ? shared_levels(ki, k(i + n_leaf)) : -1;
    const int b = min(GNB_MAXLEV, max(a, q + 1));
    int grp = 0;
    if (n_g > 0) {
        const int g = i + n_g < n ? shared_levels(ki, k(i + n_g)) : -1;
        const int lg = min(b, max(a, g + 1));
        if (lg > a || a == 0 || holder_gt(k, n, i, a - 1, n_g)) grp = lg + 1;
    }
    return (1 << 24) | (grp << 16) | (b << 8) | a;
}

__device__ __forceinline__ bool span_has(int sp, int l)
{
    if (!(sp >> 24)) return false;
    if (l == TB_NCNT - 1) return ((sp >> 16) & 255) != 0;
    return (sp & 255) <= l && l <= ((sp >> 8) & 255);
}

// Pass 1: spans, and per tile the nodes of each level and the groups.
__global__ void __launch_bounds__(TB_THREADS) k_tb_span(const uint64_t *__restrict__ k, int n, int n_leaf, int n_g,
                                                        int *__restrict__ span, int *__restrict__ tcnt, int ntiles)
{
    __shared__ int cnt[TB_NCNT];
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid < TB_NCNT) cnt[tid] = 0;
    const int base = blockIdx.x * TB_TILE;
    const KeyWin kw{k};
    __syncthreads();
    for (int r = 0; r < TB_ITEMS; r++) {
        const int i = base + r * TB_THREADS + tid;
        int sp = 0;
        if (i < n) {
            sp = span_of(kw, n, i, n_leaf, n_g);
            span[i] = sp;
        }
        // the levels present in the warp, then the groups
        const int l0 = __reduce_min_sync(0xffffffffu, (sp >> 24) ? (sp & 255) : TB_NCNT);
        const int l1 = __reduce_max_sync(0xffffffffu, (sp >> 24) ? ((sp >> 8) & 255) : -1);
        for (int l = l0; l <= l1; l++) {
            const unsigned m = __ballot_sync(0xffffffffu, span_has(sp, l));
            if (lane == 0 && m) atomicAdd(&cnt[l], __popc(m));
        }
        const unsigned m = __ballot_sync(0xffffffffu, span_has(sp, TB_NCNT - 1));
        if (lane == 0 && m) atomicAdd(&cnt[TB_NCNT - 1], __popc(m));
    }
    __syncthreads();
    if (tid < TB_NCNT) tcnt[tid * ntiles + blockIdx.x] = cnt[tid];
}

// Pass 2, one block per counter: exclusive scan over the tiles in place, and
// the counter's total.
__global__ void __launch_bounds__(1024) k_tb_scan(int *__restrict__ tcnt, int ntiles, int *__restrict__ tot)
{
    __shared__ int ws[32];
    __shared__ int s_carry;
    const int t = threadIdx.x;
    int *row = tcnt + (size_t)blockIdx.x * ntiles;
    if (t == 0) s_carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < ntiles; b0 += 1024) {
        const int i = b0 + t;
        const int v = i < ntiles ? row[i] : 0;
        int total;
        const int e = block_excl_scan(v, ws, &total);
        if (i < ntiles) row[i] = s_carry + e;
        __syncthreads();
        if (t == 0) s_carry += total;
        __syncthreads();
    }
    if (t == 0) tot[blockIdx.x] = s_carry;
}

// Pass 3: every slot writes the nodes it starts.  A node's index is its
// level's start + the tile's offset + the warps and lanes before it (ballots
// per level, kept for the round), so a slot also knows the index of its own
// node one level down -- the node's first child -- and of its own node one
// level up, the parent of every node but its first.  A node that is its
// parent's first child records the parent in head[]; the others record -1.
// Pass 4 gives every node the parent of the nearest first child at or before
// it (siblings are contiguous, at most eight) and every parent its child
// count; pass 5 the particle counts.
struct EmitShared {
    int lstart[TB_NCNT];                 // first index of each level (groups: 0)
    int run[TB_NCNT];                    // this tile's nodes so far, per counter
    int woff[TB_NCNT][TB_THREADS / 32];  // per-warp offsets of the round
    unsigned bal[TB_NCNT][TB_THREADS / 32];
    int ok;
};

__device__ void emit_slot(const Tree &t, const uint64_t *__restrict__ k, int i, int sp, const EmitShared &S, int w,
                          unsigned lt)
{
    const int a = sp & 255, b = (sp >> 8) & 255, gl = ((sp >> 16) & 255) - 1;
    const uint64_t ki = k[i];
    const int ex = compact3(ki >> 2), ey = compact3(ki >> 1), ez = compact3(ki);
    int idx = S.lstart[a] + S.woff[a][w] + __popc(S.bal[a][w] & lt);
    int parent = -1;  // the slot's first node is not a first child: pass 4 finds its parent
    for (int l = a; l <= b; l++) {
        const int sh = GNB_MAXLEV - l;
        const int child = l < b ? S.lstart[l + 1] + S.woff[l + 1][w] + __popc(S.bal[l + 1][w] & lt) : -1;
        t.head[idx] = parent;
        t.nb[idx] = make_int4((ex >> sh) << sh, (ey >> sh) << sh, (ez >> sh) << sh, parent);
        t.na[idx] = make_int4(i, 0, child, ((l < b ? 1 : 0) << 8) | l);
        if (l == gl) t.groups[S.woff[TB_NCNT - 1][w] + __popc(S.bal[TB_NCNT - 1][w] & lt)] = idx;
        parent = idx;
        idx = child;
    }
}

__global__ void __launch_bounds__(TB_THREADS) k_tb_emit(Tree t, const uint64_t *__restrict__ k, int n,
                                                        const int *__restrict__ span, const int *__restrict__ tcnt,
                                                        const int *__restrict__ tot, int ntiles,
                                                        int *__restrict__ status)
{
    __shared__ EmitShared S;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) {
        int s = 0;
        for (int l = 0; l < TB_NCNT - 1; l++) {
            S.lstart[l] = s;
            s += tot[l];
        }
        S.lstart[TB_NCNT - 1] = 0;
        S.ok = s <= t.cap;
        if (blockIdx.x == 0) {
            if (s > t.cap) {
                atomicOr(status, ST_TREE_OVERFLOW);
            } else {
                for (int l = 0; l < TB_NCNT - 1; l++) t.lvl[l] = S.lstart[l];
                t.lvl[TB_NCNT - 1] = s;
                *t.ngroups_d = tot[TB_NCNT - 1];
            }
        }
    }
    if (tid < TB_NCNT) S.run[tid] = tcnt[tid * ntiles + blockIdx.x];
    __syncthreads();
    if (!S.ok) return;
    const unsigned lt = (1u << lane) - 1u;
    const int base = blockIdx.x * TB_TILE;
    for (int r = 0; r < TB_ITEMS; r++) {
        const int i = base + r * TB_THREADS + tid;
        const int sp = i < n ? span[i] : 0;
        if (lane < TB_NCNT) {
            S.bal[lane][w] = 0u;
            S.woff[lane][w] = 0;
        }
        __syncwarp();
        const int l0 = __reduce_min_sync(0xffffffffu, (sp >> 24) ? (sp & 255) : TB_NCNT);
        const int l1 = __reduce_max_sync(0xffffffffu, (sp >> 24) ? ((sp >> 8) & 255) : -1);
        for (int l = l0; l <= l1; l++) {
            const unsigned m = __ballot_sync(0xffffffffu, span_has(sp, l));
            if (lane == 0) {
                S.bal[l][w] = m;
                S.woff[l][w] = __popc(m);
            }
        }
        {
            const unsigned m = __ballot_sync(0xffffffffu, span_has(sp, TB_NCNT - 1));
            if (lane == 0) {
                S.bal[TB_NCNT - 1][w] = m;
                S.woff[TB_NCNT - 1][w] = __popc(m);
            }
        }
        __syncthreads();
        if (tid < TB_NCNT) {
            int s = S.run[tid];
            for (int q = 0; q < TB_THREADS / 32; q++) {
                const int c = S.woff[tid][q];
                S.woff[tid][q] = s;
                s += c;
            }
            S.run[tid] = s;
        }
        __syncthreads();
        if (sp >> 24) emit_slot(t, k, i, sp, S, w, lt);
        __syncthreads();
    }
}

// Pass 4, per node: the parent is the head of the nearest first child at or
// before the node; the last of a parent's children (the next node is a first
// child, or there is none) writes the parent's child count.
__global__ void __launch_bounds__(TB_THREADS) k_tb_link(Tree t, int nn)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k <= 0 || k >= nn) return;  // the root has no parent
    int j = k, p = t.head[k];
    while (p < 0 && j > 0) p = t.head[--j];
    reinterpret_cast<int *>(&t.nb[k])[3] = p;
    if (k + 1 == nn || t.head[k + 1] >= 0) {
        const int4 pa = t.na[p];
        reinterpret_cast<int *>(&t.na[p])[3] = ((k - pa.z + 1) << 8) | (pa.w & 255);
    }
}

// Pass 5, per node: its cell ends where its next sibling starts; a last
// child ends with its parent (up to the root, which ends at n).
__global__ void __launch_bounds__(TB_THREADS) k_tb_count(Tree t, int n, int nn)
{
    const int node = blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= nn) return;
    int cur = node, end = n;
    for (;;) {
        const int p = t.nb[cur].w;
        if (p < 0) break;
        const int4 pa = t.na[p];
        if (cur != pa.z + (pa.w >> 8) - 1) {
            end = t.na[cur + 1].x;
            break;
        }
        cur = p;
    }
    t.na[node].y = end - t.na[node].x;
}

// ----------------------------------------------------------------- moments
// Four lanes per node: a leaf's lanes take four of its particles each per
// round (the loads of a round issued together), an inner node's lanes two of
// its children each, and the sums are shuffle reductions over the four
// lanes.  All leaves in one launch, then the inner nodes one level at a time
// from the deepest up (a parent combines its children with the
// parallel-axis shift).
struct PartView {
    const int *cx, *cy, *cz;
    const float *rx, *ry, *rz, *m, *eps;
};

#define MO_LANES 4

__device__ __forceinline__ float sum4(float v, unsigned gm)
{
    v += __shfl_xor_sync(gm, v, 2, MO_LANES);
    v += __shfl_xor_sync(gm, v, 1, MO_LANES);
    return v;
}

__device__ __forceinline__ void store_moments(const Tree &t, int node, float cx, float cy, float cz, float M,
                                              const float q[6], float e2)
{
    t.mo0[node] = make_float4(cx, cy, cz, M);
    t.mo1[node] = make_float4(q[0], q[1], q[2], q[3]);
    t.mo2[node] = make_float4(q[4], q[5], e2, 0.f);
}

__global__ void __launch_bounds__(TB_THREADS) k_moments_leaf(Tree t, int nn, PartView p, const double *__restrict__ box)
{
    const float unit = (float)box[4];
    const int lane = threadIdx.x & 31, g = lane & (MO_LANES - 1);
    const unsigned gm = 0xfu << (lane & ~(MO_LANES - 1));
    const int stride = (gridDim.x * blockDim.x) / MO_LANES;
    for (int node = (blockIdx.x * blockDim.x + threadIdx.x) / MO_LANES; node < nn; node += stride) {
        const int4 a = t.na[node];
        if ((a.w >> 8) != 0) continue;  // an inner node
        const int4 C = t.nb[node];
        const int end = a.x + a.y;
        float M = 0.f, sx = 0.f, sy = 0.f, sz = 0.f, se = 0.f;
        for (int j0 = a.x + g; j0 < end; j0 += 4 * MO_LANES) {
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const int j = j0 + r * MO_LANES;
                if (j < end) {
                    const float mj = p.m[j];
                    M += mj;
                    sx += mj * grid_off(p.cx[j], C.x, p.rx[j], unit);
                    sy += mj * grid_off(p.cy[j], C.y, p.ry[j], unit);
                    sz += mj * grid_off(p.cz[j], C.z, p.rz[j], unit);
                    se += mj * p.eps[j] * p.eps[j];
                }
            }
        }
        M = sum4(M, gm);
        const float cx = sum4(sx, gm) / M, cy = sum4(sy, gm) / M, cz = sum4(sz, gm) / M;
        se = sum4(se, gm);
        float q[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int j0 = a.x + g; j0 < end; j0 += 4 * MO_LANES) {
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const int j = j0 + r * MO_LANES;
                if (j < end) {
                    const float mj = p.m[j];
                    const float dx = grid_off(p.cx[j], C.x, p.rx[j], unit) - cx;
                    const float dy = grid_off(p.cy[j], C.y, p.ry[j], unit) - cy;
                    const float dz = grid_off(p.cz[j], C.z, p.rz[j], unit) - cz;
                    const float dd = dx * dx + dy * dy + dz * dz;
                    q[0] += mj * (3.f * dx * dx - dd);
                    q[1] += mj * (3.f * dy * dy - dd);
                    q[2] += mj * (3.f * dz * dz - dd);
                    q[3] += mj * 3.f * dx * dy;
                    q[4] += mj * 3.f * dx * dz;
                    q[5] += mj * 3.f * dy * dz;
                }
            }
        }
#pragma unroll
        for (int r = 0; r < 6; r++) q[r] = sum4(q[r], gm);
        if (g == 0) store_moments(t, node, cx, cy, cz, M, q, se / M);
    }
}

// the inner nodes of [b, e) (one level)
__global__ void __launch_bounds__(TB_THREADS) k_moments_inner(Tree t, int b, int e, const double *__restrict__ box)
{
    const float unit = (float)box[4];
    const int lane = threadIdx.x & 31, g = lane & (MO_LANES - 1);
    const unsigned gm = 0xfu << (lane & ~(MO_LANES - 1));
    const int stride = (gridDim.x * blockDim.x) / MO_LANES;
    for (int node = b + (blockIdx.x * blockDim.x + threadIdx.x) / MO_LANES; node < e; node += stride) {
        const int4 a = t.na[node];
        const int nch = a.w >> 8;
        if (nch == 0) continue;  // a leaf
        const int4 P = t.nb[node];
        float4 m0[2], m1[2], m2[2];
        float ox[2], oy[2], oz[2];
#pragma unroll
        for (int r = 0; r < 2; r++) {
            const int c = g + r * MO_LANES;
            m0[r] = m1[r] = m2[r] = make_float4(0.f, 0.f, 0.f, 0.f);
            ox[r] = oy[r] = oz[r] = 0.f;
            if (c < nch) {
                m0[r] = t.mo0[a.z + c];
                m1[r] = t.mo1[a.z + c];
                m2[r] = t.mo2[a.z + c];
                const int4 Cc = t.nb[a.z + c];
                ox[r] = (float)(Cc.x - P.x) * unit + m0[r].x;
                oy[r] = (float)(Cc.y - P.y) * unit + m0[r].y;
                oz[r] = (float)(Cc.z - P.z) * unit + m0[r].z;
            }
        }
        const float M = sum4(m0[0].w + m0[1].w, gm);
        const float cx = sum4(m0[0].w * ox[0] + m0[1].w * ox[1], gm) / M;
        const float cy = sum4(m0[0].w * oy[0] + m0[1].w * oy[1], gm) / M;
        const float cz = sum4(m0[0].w * oz[0] + m0[1].w * oz[1], gm) / M;
        const float se = sum4(m0[0].w * m2[0].z + m0[1].w * m2[1].z, gm);
        float q[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int r = 0; r < 2; r++) {
            const float mc = m0[r].w;
            const float dx = ox[r] - cx, dy = oy[r] - cy, dz = oz[r] - cz;
            const float dd = dx * dx + dy * dy + dz * dz;
            q[0] += m1[r].x + mc * (3.f * dx * dx - dd);
            q[1] += m1[r].y + mc * (3.f * dy * dy - dd);
            q[2] += m1[r].z + mc * (3.f * dz * dz - dd);
            q[3] += m1[r].w + mc * 3.f * dx * dy;
            q[4] += m2[r].x + mc * 3.f * dx * dz;
            q[5] += m2[r].y + mc * 3.f * dy * dz;
        }
#pragma unroll
        for (int r = 0; r < 6; r++) q[r] = sum4(q[r], gm);
        if (g == 0) store_moments(t, node, cx, cy, cz, M, q, se / M);
    }
}

// ----------------------------------------------------------------- host
int tree_alloc(gnb_ctx *c, Tree &t, int cap)
{
    // node arrays only; the per-slot scratch survives a regrow
    dfree(c, t.na); dfree(c, t.nb); dfree(c, t.mo0); dfree(c, t.mo1); dfree(c, t.mo2); dfree(c, t.head);
    t.cap = cap;
    GNB_TRY(dalloc(c, &t.na, cap));
    GNB_TRY(dalloc(c, &t.nb, cap));
    GNB_TRY(dalloc(c, &t.mo0, cap));
    GNB_TRY(dalloc(c, &t.mo1, cap));
    GNB_TRY(dalloc(c, &t.mo2, cap));
    GNB_TRY(dalloc(c, &t.head, cap));
    return GNB_OK;
}

static int tree_scratch(gnb_ctx *c, Tree &t, int n, int ntiles)
{
    if (!t.lvl) {
        GNB_TRY(dalloc(c, &t.lvl, GNB_MAXLEV + 4));
        GNB_TRY(dalloc(c, &t.tot, TB_NCNT));
        GNB_TRY(dalloc(c, &t.ngroups_d, 4));
    }
    if (n + 1 > t.scap) {
        dfree(c, t.span); dfree(c, t.groups);
        GNB_TRY(dalloc(c, &t.span, (size_t)n + 1));
        GNB_TRY(dalloc(c, &t.groups, (size_t)n + 1));
        t.scap = n + 1;
    }
    if (ntiles * TB_NCNT > t.tcap) {
        dfree(c, t.tcnt);
        GNB_TRY(dalloc(c, &t.tcnt, (size_t)ntiles * TB_NCNT));
        t.tcap = ntiles * TB_NCNT;
    }
    return GNB_OK;
}

void tree_free(gnb_ctx *c, Tree &t)
{
    dfree(c, t.na); dfree(c, t.nb); dfree(c, t.mo0); dfree(c, t.mo1); dfree(c, t.mo2); dfree(c, t.head);
    dfree(c, t.lvl); dfree(c, t.tot); dfree(c, t.ngroups_d); dfree(c, t.span); dfree(c, t.groups);
    dfree(c, t.tcnt);
    t = Tree();
}

// Build the tree over n >= 1 sorted keys: the node array, the groups of at
// most n_group particles (none when n_group <= 0) and, optionally, the
// moments.  Six launches whatever the depth, the moments one per level, and
// one wait on the stream, for the node count and the level table.
int build_tree(gnb_ctx *c, Tree &t, const uint64_t *skey, int n, const int *n_d, int n_leaf, int n_group,
               const int *pcx, const int *pcy, const int *pcz, const float *prx, const float *pry, const float *prz,
               const float *pm, const float *peps, bool moments)
{
    (void)n_d;
    if (n <= 0) return fail(c, GNB_EINVAL, "tree over no particles");
    const int ntiles = (n + TB_TILE - 1) / TB_TILE;
    GNB_TRY(tree_scratch(c, t, n, ntiles));
    if (t.cap < 64) GNB_TRY(tree_alloc(c, t, n + n / 2 + 1024));
    gnb::counted(k_tb_span)<<<ntiles, TB_THREADS, 0, c->s>>>(skey, n, n_leaf, n_group, t.span, t.tcnt, ntiles);
    gnb::counted(k_tb_scan)<<<TB_NCNT, 1024, 0, c->s>>>(t.tcnt, ntiles, t.tot);
    const int *lv = c->pinned_i + 1;  // level table copy [GNB_MAXLEV + 2]
    for (int attempt = 0;; attempt++) {
        gnb::counted(k_tb_emit)<<<ntiles, TB_THREADS, 0, c->s>>>(t, skey, n, t.span, t.tcnt, t.tot, ntiles,
                                                                  c->status_d);
        GNB_LAUNCH_CHECK(c, "tree build");
        cudaMemcpyAsync(c->pinned_i, c->status_d, sizeof(int), cudaMemcpyDeviceToHost, c->s);
        cudaMemcpyAsync(c->pinned_i + 1, t.lvl, sizeof(int) * (GNB_MAXLEV + 2), cudaMemcpyDeviceToHost, c->s);
        GNB_TRY(cuda_check(c, cudaStreamSynchronize(c->s), "tree build sync"));
        if (!(c->pinned_i[0] & ST_TREE_OVERFLOW)) break;
        if (attempt > 0) return fail(c, GNB_ECAPACITY, "tree node capacity");
        // more nodes than the arrays hold: grow them to the count and emit again
        int tot_h[TB_NCNT];
        GNB_TRY(cuda_check(c, cudaMemcpy(tot_h, t.tot, sizeof(tot_h), cudaMemcpyDeviceToHost), "node count"));
        long long need = 0;
        for (int l = 0; l < TB_NCNT - 1; l++) need += tot_h[l];
        const int zero = 0;
        GNB_TRY(cuda_check(c, cudaMemcpy(c->status_d, &zero, sizeof(int), cudaMemcpyHostToDevice), "status reset"));
        if (need + need / 4 + 1024 > INT32_MAX) return fail(c, GNB_ECAPACITY, "tree node capacity");
        GNB_TRY(tree_alloc(c, t, (int)(need + need / 4 + 1024)));
    }
    t.nnodes = lv[GNB_MAXLEV + 1];
    t.depth = 0;
    for (int l = 0; l <= GNB_MAXLEV; l++)
        if (lv[l + 1] > lv[l]) t.depth = l;
    if (t.nnodes <= 0) return fail(c, GNB_ECAPACITY, "tree node capacity");
    gnb::counted(k_tb_link)<<<(t.nnodes + TB_THREADS - 1) / TB_THREADS, TB_THREADS, 0, c->s>>>(t, t.nnodes);
    gnb::counted(k_tb_count)<<<(t.nnodes + TB_THREADS - 1) / TB_THREADS, TB_THREADS, 0, c->s>>>(t, n, t.nnodes);
    GNB_LAUNCH_CHECK(c, "tree links");
    if (moments) {
        PartView p{pcx, pcy, pcz, prx, pry, prz, pm, peps};
        auto blocks = [&](long long nodes) {
            return (int)std::max(1ll, std::min((nodes * MO_LANES + TB_THREADS - 1) / TB_THREADS, 152ll * 64));
        };
        gnb::counted(k_moments_leaf)<<<blocks(t.nnodes), TB_THREADS, 0, c->s>>>(t, t.nnodes, p, c->box_d);
        for (int l = t.depth - 1; l >= 0; l--)  // the deepest level holds leaves only
            gnb::counted(k_moments_inner)<<<blocks(lv[l + 1] - lv[l]), TB_THREADS, 0, c->s>>>(t, lv[l], lv[l + 1],
                                                                                               c->box_d);
        GNB_LAUNCH_CHECK(c, "moments");
    }
    return GNB_OK;
}

}  // namespace gnb
