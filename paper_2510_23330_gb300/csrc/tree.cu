// tree.cu -- octree over Morton-sorted particles, cell moments and groups
// (Barnes-Hut treecode, Sec. 1 and 3.4; groups sharing one interaction list,
// Sec. 5.2.2 and 5.2.4 of Hirashima et al., SC'25).
//
// A level-l cell holds the particles sharing the top 3l key bits.  A cell is
// split when it holds more than n_leaf particles and l < 21; its non-empty
// children are stored in Morton order.  The build runs one level at a time
// entirely on the device (split count, scan of the per-block child counts,
// emission), so the node array is the breadth-first list and the host never
// waits on it.  Level bounds live in t.lvl: level l is [lvl[l], lvl[l+1]).
//
// Moments are FP32 about each cell's integer corner: M, centre of mass
// offset, traceless quadrupole Q = sum m (3 d d - d^2 I) about the centre of
// mass, and the mass-weighted mean eps^2.  Parents combine their children
// with the parallel-axis shift.
#include "common.cuh"

namespace gnb {

#define TB_THREADS 256
#define TB_BLOCKS 304

// ----------------------------------------------------------------- scan
__global__ void k_scan_partial(const int *__restrict__ in, const int *__restrict__ n_d, int *partial)
{
    __shared__ int ws[32];
    int n = *n_d, G = gridDim.x;
    int chunk = (n + G - 1) / G;
    int beg = blockIdx.x * chunk, end = min(n, beg + chunk);
    int s = 0;
    for (int i = beg + threadIdx.x; i < end; i += blockDim.x) s += in[i];
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
    int chunk = (n + G - 1) / G;
    int beg = blockIdx.x * chunk, end = min(n, beg + chunk);
    int carry = poff[blockIdx.x];
    for (int b0 = beg; b0 < end; b0 += blockDim.x) {
        int i = b0 + threadIdx.x;
        int v = i < end ? in[i] : 0;
        int tot;
        int e = block_excl_scan(v, ws, &tot);
        if (i < end) out[i] = carry + e;
        carry += tot;
    }
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
__global__ void k_tree_root(Tree t, int n)
{
    int i = threadIdx.x;
    if (i == 0) {
        t.na[0] = make_int4(0, n, -1, 0);
        t.nb[0] = make_int4(0, 0, 0, -1);
    }
    if (i <= GNB_MAXLEV + 1) t.lvl[i] = (i == 0) ? 0 : 1;
}

// First slot in [b, e) whose key is >= target.
__device__ __forceinline__ int lower_bound_key(const uint64_t *__restrict__ k, int b, int e, uint64_t target)
{
    while (b < e) {
        int m = (b + e) >> 1;
        if (k[m] < target) b = m + 1;
        else e = m;
    }
    return b;
}

// pos[d] = first slot of child digit d (pos[8] = end) of a level-l cell.
__device__ __forceinline__ void child_bounds(const uint64_t *__restrict__ k, int first, int count, int l,
                                             int pos[9])
{
    int sh = 3 * (GNB_MAXLEV - (l + 1));
    uint64_t base = (k[first] >> (sh + 3)) << (sh + 3);
    pos[0] = first;
    pos[8] = first + count;
#pragma unroll
    for (int d = 1; d < 8; d++) pos[d] = lower_bound_key(k, pos[d - 1], first + count, base | ((uint64_t)d << sh));
}

// ptab[c] = first slot whose key is >= prefix c at level GNB_PTAB_LEVEL
// (c < 8^L), ptab[8^L] = n: independent binary searches, all in parallel.
__global__ void k_prefix_table(const uint64_t *__restrict__ k, int n, int *__restrict__ ptab)
{
    const int ncell = 1 << (3 * GNB_PTAB_LEVEL);
    const int sh = 3 * (GNB_MAXLEV - GNB_PTAB_LEVEL);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= ncell; c += gridDim.x * blockDim.x)
        ptab[c] = c == ncell ? n : lower_bound_key(k, 0, n, (uint64_t)c << sh);
}

__global__ void __launch_bounds__(TB_THREADS) k_split_count(Tree t, const uint64_t *__restrict__ k, int l,
                                                            int n_leaf)
{
    __shared__ int ws[32];
    int lb = t.lvl[l], le = t.lvl[l + 1];
    int nl = le - lb, G = gridDim.x;
    int chunk = (nl + G - 1) / G;
    int beg = lb + blockIdx.x * chunk, end = min(le, beg + chunk);
    // eight lanes per node, lane d finds the first slot of child digit d, so
    // the seven binary searches of a node run side by side
    const int d = threadIdx.x & 7;
    const int sh = 3 * (GNB_MAXLEV - (l + 1));
    int s = 0;
    for (int b0 = beg; b0 < end; b0 += blockDim.x >> 3) {
        int node = b0 + (threadIdx.x >> 3);
        bool live = node < end;
        int4 a = live ? t.na[node] : make_int4(0, 0, 0, 0);
        bool split = live && a.y > n_leaf && l < GNB_MAXLEV;
        int pos = a.x;
        if (split && d > 0) {
            uint64_t base = (k[a.x] >> (sh + 3)) << (sh + 3);
            const uint64_t target = base | ((uint64_t)d << sh);
            // a node's keys share its prefix, so the first slot >= target in
            // the whole array lies in [a.x, a.x + a.y]: the table's entry
            if (l < GNB_PTAB_LEVEL) pos = t.ptab[target >> (3 * (GNB_MAXLEV - GNB_PTAB_LEVEL))];
            else pos = lower_bound_key(k, a.x, a.x + a.y, target);
        }
        int nxt = __shfl_down_sync(0xffffffffu, pos, 1, 8);
        if (d == 7) nxt = a.x + a.y;
        unsigned ne = __ballot_sync(0xffffffffu, split && nxt > pos);
        int nch = __popc((ne >> (threadIdx.x & 24)) & 0xffu);
        if (split) t.cb[(size_t)node * 8 + d] = pos;
        if (live && d == 0) {
            t.na[node].w = (nch << 8) | l;
            s += nch;
        }
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        int v = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0;
        v = warp_sum(v);
        if (threadIdx.x == 0) t.partial[blockIdx.x] = v;
    }
}

__global__ void k_level_scan(Tree t, int l, int G, int *status)
{
    __shared__ int ws[32];
    int th = threadIdx.x, lane = th & 31, w = th >> 5;
    int v = th < G ? t.partial[th] : 0;
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
    if (th < G) t.poff[th] = x - v + (w > 0 ? ws[w - 1] : 0);
    if (th == 0) {
        int total = ws[31];
        int le = t.lvl[l + 1];
        if ((long long)le + total > (long long)t.cap) {
            atomicOr(status, ST_TREE_OVERFLOW);
            total = 0;
        }
        t.poff[G] = total;
        for (int q = l + 2; q <= GNB_MAXLEV + 1; q++) t.lvl[q] = le + total;
    }
}

__global__ void __launch_bounds__(TB_THREADS) k_emit(Tree t, const uint64_t *__restrict__ k, int l)
{
    __shared__ int ws[32];
    int lb = t.lvl[l], le = t.lvl[l + 1];
    int G = gridDim.x;
    if (t.poff[G] == 0) return;
    int nl = le - lb;
    int chunk = (nl + G - 1) / G;
    int beg = lb + blockIdx.x * chunk, end = min(le, beg + chunk);
    int carry = le + t.poff[blockIdx.x];
    int side = 1 << (GNB_MAXLEV - (l + 1));
    // eight lanes per node (lane d = child digit d), 32 nodes per iteration
    __shared__ int s_n[32], s_ex[33];
    const int d = threadIdx.x & 7, j = threadIdx.x >> 3;
    (void)ws;
    for (int b0 = beg; b0 < end; b0 += blockDim.x >> 3) {
        int node = b0 + j;
        bool live = node < end;
        int4 a = live ? t.na[node] : make_int4(0, 0, 0, 0);
        int nch = live ? (a.w >> 8) : 0;
        int pos = nch > 0 ? t.cb[(size_t)node * 8 + d] : 0;
        int nxt = __shfl_down_sync(0xffffffffu, pos, 1, 8);
        if (d == 7) nxt = a.x + a.y;
        bool ne = nch > 0 && nxt > pos;
        unsigned bal = __ballot_sync(0xffffffffu, ne);
        unsigned mine = (bal >> (threadIdx.x & 24)) & 0xffu;
        if (d == 0) s_n[j] = nch;
        __syncthreads();
        if (threadIdx.x < 32) {
            int v = s_n[threadIdx.x], x = v;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, x, o);
                if (threadIdx.x >= o) x += y;
            }
            s_ex[threadIdx.x] = x - v;
            if (threadIdx.x == 31) s_ex[32] = x;
        }
        __syncthreads();
        int base = carry + s_ex[j];
        if (nch > 0 && d == 0) t.na[node].z = base;
        if (ne) {
            int q = __popc(mine & ((1u << d) - 1u));
            int4 cbn = t.nb[node];
            t.na[base + q] = make_int4(pos, nxt - pos, -1, l + 1);
            t.nb[base + q] = make_int4(cbn.x + ((d >> 2) & 1) * side, cbn.y + ((d >> 1) & 1) * side,
                                       cbn.z + (d & 1) * side, node);
        }
        carry += s_ex[32];
        __syncthreads();
    }
}

// ----------------------------------------------------------------- moments
__global__ void k_moments_level(Tree t, int l, const int *__restrict__ pcx, const int *__restrict__ pcy,
                                const int *__restrict__ pcz, const float *__restrict__ prx,
                                const float *__restrict__ pry, const float *__restrict__ prz,
                                const float *__restrict__ pm, const float *__restrict__ peps,
                                const double *__restrict__ box)
{
    int lb = t.lvl[l], le = t.lvl[l + 1];
    float unit = (float)box[4];
    for (int node = lb + blockIdx.x * blockDim.x + threadIdx.x; node < le; node += gridDim.x * blockDim.x) {
        int4 a = t.na[node];
        int4 C = t.nb[node];
        int nch = a.w >> 8;
        float M = 0.f, sx = 0.f, sy = 0.f, sz = 0.f, se = 0.f;
        float q0 = 0.f, q1 = 0.f, q2 = 0.f, q3 = 0.f, q4 = 0.f, q5 = 0.f;
        if (nch == 0) {
            for (int j = a.x; j < a.x + a.y; j++) {
                float mj = pm[j];
                float ox = grid_off(pcx[j], C.x, prx[j], unit);
                float oy = grid_off(pcy[j], C.y, pry[j], unit);
                float oz = grid_off(pcz[j], C.z, prz[j], unit);
                M += mj;
                sx += mj * ox; sy += mj * oy; sz += mj * oz;
                se += mj * peps[j] * peps[j];
            }
            float cx = sx / M, cy = sy / M, cz = sz / M;
            for (int j = a.x; j < a.x + a.y; j++) {
                float mj = pm[j];
                float dx = grid_off(pcx[j], C.x, prx[j], unit) - cx;
                float dy = grid_off(pcy[j], C.y, pry[j], unit) - cy;
                float dz = grid_off(pcz[j], C.z, prz[j], unit) - cz;
                float dd = dx * dx + dy * dy + dz * dz;
                q0 += mj * (3.f * dx * dx - dd);
                q1 += mj * (3.f * dy * dy - dd);
                q2 += mj * (3.f * dz * dz - dd);
                q3 += mj * 3.f * dx * dy;
                q4 += mj * 3.f * dx * dz;
                q5 += mj * 3.f * dy * dz;
            }
            t.mo0[node] = make_float4(cx, cy, cz, M);
            t.mo1[node] = make_float4(q0, q1, q2, q3);
            t.mo2[node] = make_float4(q4, q5, se / M, 0.f);
        } else {
            for (int c = a.z; c < a.z + nch; c++) {
                float4 m0 = t.mo0[c];
                float4 m2 = t.mo2[c];
                int4 Cc = t.nb[c];
                float ox = (float)(Cc.x - C.x) * unit + m0.x;
                float oy = (float)(Cc.y - C.y) * unit + m0.y;
                float oz = (float)(Cc.z - C.z) * unit + m0.z;
                M += m0.w;
                sx += m0.w * ox; sy += m0.w * oy; sz += m0.w * oz;
                se += m0.w * m2.z;
            }
            float cx = sx / M, cy = sy / M, cz = sz / M;
            for (int c = a.z; c < a.z + nch; c++) {
                float4 m0 = t.mo0[c];
                float4 m1 = t.mo1[c];
                float4 m2 = t.mo2[c];
                int4 Cc = t.nb[c];
                float dx = (float)(Cc.x - C.x) * unit + m0.x - cx;
                float dy = (float)(Cc.y - C.y) * unit + m0.y - cy;
                float dz = (float)(Cc.z - C.z) * unit + m0.z - cz;
                float dd = dx * dx + dy * dy + dz * dz;
                float mc = m0.w;
                q0 += m1.x + mc * (3.f * dx * dx - dd);
                q1 += m1.y + mc * (3.f * dy * dy - dd);
                q2 += m1.z + mc * (3.f * dz * dz - dd);
                q3 += m1.w + mc * 3.f * dx * dy;
                q4 += m2.x + mc * 3.f * dx * dz;
                q5 += m2.y + mc * 3.f * dy * dz;
            }
            t.mo0[node] = make_float4(cx, cy, cz, M);
            t.mo1[node] = make_float4(q0, q1, q2, q3);
            t.mo2[node] = make_float4(q4, q5, se / M, 0.f);
        }
    }
}

// ----------------------------------------------------------------- groups
// A group is a cell with count <= n_g, or a leaf, whose parent has more than
// n_g particles (the first such cell on every root-to-leaf path).
__global__ void k_group_mark(Tree t, int n_group, int *__restrict__ mark)
{
    int nn = t.lvl[GNB_MAXLEV + 1];
    for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < nn; node += gridDim.x * blockDim.x) {
        int4 a = t.na[node];
        int nch = a.w >> 8;
        bool g = (a.y <= n_group || nch == 0);
        if (g && node > 0) {
            int par = t.nb[node].w;
            g = t.na[par].y > n_group;
        }
        if (g) mark[a.x] = node;
    }
}

__global__ void k_group_flag(const int *__restrict__ mark, int *__restrict__ flag, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = mark[i] >= 0;
}

__global__ void k_group_compact(const int *__restrict__ mark, const int *__restrict__ off, int n,
                                int *__restrict__ groups)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && mark[i] >= 0) groups[off[i]] = mark[i];
}

int tree_alloc(gnb_ctx *c, Tree &t, int cap)
{
    // node arrays only; the per-particle group scratch survives a regrow
    dfree(c, t.na); dfree(c, t.nb); dfree(c, t.mo0); dfree(c, t.mo1); dfree(c, t.mo2); dfree(c, t.cb);
    dfree(c, t.lvl); dfree(c, t.partial); dfree(c, t.poff); dfree(c, t.ngroups_d); dfree(c, t.ptab);
    t.cap = cap;
    GNB_TRY(dalloc(c, &t.na, cap));
    GNB_TRY(dalloc(c, &t.nb, cap));
    GNB_TRY(dalloc(c, &t.mo0, cap));
    GNB_TRY(dalloc(c, &t.mo1, cap));
    GNB_TRY(dalloc(c, &t.mo2, cap));
    GNB_TRY(dalloc(c, &t.cb, (size_t)cap * 8));
    GNB_TRY(dalloc(c, &t.lvl, GNB_MAXLEV + 4));
    GNB_TRY(dalloc(c, &t.partial, 1100));
    GNB_TRY(dalloc(c, &t.poff, 1100));
    GNB_TRY(dalloc(c, &t.ngroups_d, 4));
    GNB_TRY(dalloc(c, &t.ptab, ((size_t)1 << (3 * GNB_PTAB_LEVEL)) + 1));
    return GNB_OK;
}

void tree_free(gnb_ctx *c, Tree &t)
{
    dfree(c, t.na); dfree(c, t.nb); dfree(c, t.mo0); dfree(c, t.mo1); dfree(c, t.mo2); dfree(c, t.cb);
    dfree(c, t.lvl); dfree(c, t.partial); dfree(c, t.poff); dfree(c, t.gmark); dfree(c, t.gflag);
    dfree(c, t.goff); dfree(c, t.groups); dfree(c, t.ngroups_d); dfree(c, t.ptab);
    t = Tree();
}

// Build the tree over n sorted keys; optional moments.  Groups use the
// scratch arrays gflag/groups (length >= n + 1), allocated here on demand.
int build_tree(gnb_ctx *c, Tree &t, const uint64_t *skey, int n, const int *n_d, int n_leaf,
               int n_group, const int *pcx, const int *pcy, const int *pcz, const float *prx, const float *pry,
               const float *prz, const float *pm, const float *peps, bool moments)
{
    for (int attempt = 0; attempt < 6; attempt++) {
        if (t.cap < 64) GNB_TRY(tree_alloc(c, t, n + n / 2 + 1024));
        gnb::counted(k_tree_root)<<<1, 32, 0, c->s>>>(t, n);
        gnb::counted(k_prefix_table)<<<((1 << (3 * GNB_PTAB_LEVEL)) + TB_THREADS) / TB_THREADS, TB_THREADS, 0,
                                        c->s>>>(skey, n, t.ptab);  // one search per thread
        // Levels down to two below the last build's depth, then one check of
        // the overflow flag and the level table; the remaining levels run only
        // if the last level built still holds nodes (the tree got deeper).
        int from = 0, L = std::min(GNB_MAXLEV, t.depth + 2);
        bool over = false;
        const int *lv = c->pinned_i + 1;  // level table copy [GNB_MAXLEV + 2]
        for (;;) {
            for (int l = from; l < L; l++) {
                gnb::counted(k_split_count)<<<TB_BLOCKS, TB_THREADS, 0, c->s>>>(t, skey, l, n_leaf);
                gnb::counted(k_level_scan)<<<1, 1024, 0, c->s>>>(t, l, TB_BLOCKS, c->status_d);
                gnb::counted(k_emit)<<<TB_BLOCKS, TB_THREADS, 0, c->s>>>(t, skey, l);
            }
            if (L == GNB_MAXLEV) gnb::counted(k_split_count)<<<TB_BLOCKS, TB_THREADS, 0, c->s>>>(t, skey, GNB_MAXLEV, n_leaf);
            GNB_LAUNCH_CHECK(c, "tree build");
            cudaMemcpyAsync(c->pinned_i, c->status_d, sizeof(int), cudaMemcpyDeviceToHost, c->s);
            cudaMemcpyAsync(c->pinned_i + 1, t.lvl, sizeof(int) * (GNB_MAXLEV + 2), cudaMemcpyDeviceToHost, c->s);
            GNB_TRY(cuda_check(c, cudaStreamSynchronize(c->s), "tree build sync"));
            if (c->pinned_i[0] & ST_TREE_OVERFLOW) {
                over = true;
                break;
            }
            if (L == GNB_MAXLEV || lv[L + 1] == lv[L]) break;  // level L is empty: the tree is complete
            from = L;
            L = GNB_MAXLEV;
        }
        if (over) {
            int zero = 0;
            cudaMemcpyAsync(c->status_d, &zero, sizeof(int), cudaMemcpyHostToDevice, c->s);
            cudaStreamSynchronize(c->s);
            GNB_TRY(tree_alloc(c, t, t.cap * 2));
            continue;
        }
        t.nnodes = lv[GNB_MAXLEV + 1];
        t.depth = 0;
        for (int l = 0; l <= GNB_MAXLEV; l++)
            if (lv[l + 1] > lv[l]) t.depth = l;
        break;
    }
    if (t.nnodes <= 0) return fail(c, GNB_ECAPACITY, "tree node capacity");
    if (moments) {
        for (int l = t.depth; l >= 0; l--)  // deeper levels are empty
            gnb::counted(k_moments_level)<<<TB_BLOCKS, TB_THREADS, 0, c->s>>>(t, l, pcx, pcy, pcz, prx, pry, prz, pm, peps,
                                                                c->box_d);
        GNB_LAUNCH_CHECK(c, "moments");
    }
    if (n_group > 0) {
        if (!t.gmark) {
            GNB_TRY(dalloc(c, &t.gmark, (size_t)n + 1));
            GNB_TRY(dalloc(c, &t.gflag, (size_t)n + 1));
            GNB_TRY(dalloc(c, &t.goff, (size_t)n + 1));
            GNB_TRY(dalloc(c, &t.groups, (size_t)n + 1));
        }
        int nb = (n + 255) / 256;
        cudaMemsetAsync(t.gmark, 0xff, sizeof(int) * (size_t)n, c->s);
        gnb::counted(k_group_mark)<<<TB_BLOCKS, TB_THREADS, 0, c->s>>>(t, n_group, t.gmark);
        gnb::counted(k_group_flag)<<<nb, 256, 0, c->s>>>(t.gmark, t.gflag, n);
        GNB_TRY(device_scan(c, t.gflag, t.goff, n_d, n, t.ngroups_d));
        gnb::counted(k_group_compact)<<<nb, 256, 0, c->s>>>(t.gmark, t.goff, n, t.groups);
        GNB_LAUNCH_CHECK(c, "groups");
    }
    return GNB_OK;
}

}  // namespace gnb
