// gravity.cu -- softened self-gravity (Eq. 1 of Hirashima et al., SC'25)
// by Barnes-Hut group walk (Sec. 3.4, 5.2.2, 5.2.4) or direct summation,
// plus the static NFW halo of the disk model.
//
// Design (GB300), tree gravity in two kernels:
//  * k_grav_walk: one warp per group walks the octree (Sec. 3.4) with a
//    per-warp shared-memory stack, testing up to 32 nodes at a time with the
//    exact integer opening test, and writes the group's interaction lists --
//    accepted cells and opened leaves -- into chains of 256-entry chunks of a
//    device pool.  No CTA barriers, high occupancy: the walk is latency bound
//    and many warps hide the latency of the node loads.
//  * k_grav_eval: one CTA of GW_THREADS threads per group, scheduled
//    persistently; it streams the group's chains through shared memory,
//    staging accepted cells (monopole + quadrupole) and the particles of
//    opened leaves as FP32 offsets from the group's reference grid point
//    (Sec. 4.3 mixed precision); every thread evaluates its i-particles
//    (one, two above 16, four above 64 and eight above 128 particles per
//    group chunk; from two on in float2 pairs on the FP32x2 instructions)
//    against the staged j entries, read as warp-wide broadcasts, and the j
//    loop is split over as many thread sets as fit ("j-splits") so all
//    warps stay busy.
// Pair arithmetic is FP32 on the CUDA cores (not a dense contraction).
#include <algorithm>

#include "common.cuh"

namespace gnb {

#define GW_THREADS 128
#define GL_CH 256        // entries per list chunk
#define GL_WARPS 8       // warps per walk CTA
#define GL_STACK 1024    // walk stack entries per warp
#define GW_LEAF 256
#define GW_JP 512
#define GW_JC 256

struct GravParams {
    int4 *na, *nb;
    float4 *mo0, *mo1, *mo2;
    const int *groups, *ngroups;
    const int *cx, *cy, *cz;
    const float *rx, *ry, *rz, *m, *eps;
    float *ax, *ay, *az, *pot;
    const double *box;
    double theta2;
    long long open_d2max[GNB_MAXLEV + 1];  // per level: largest d2 that opens a cell (see must_open)
    float G;
    float e2u;  // 2 fl(eps^2) when every particle has the same softening eps > 0
    int quad;
    int n;
    int *next;
    int *status;
    unsigned long long *counters;
    // interaction-list pool (tree walk -> evaluation)
    int *pool, *cnext, *ccnt, *top;
    int *lcum;     // leaf chains: offset of each leaf's first particle in the group's leaf-particle list
    int4 *ghead;   // per group: {cell chain head, leaf chain head, particles in opened leaves, -}
    int4 *gref;    // per group: reference grid cell {x, y, z, -}
    int cap;       // pool chunks
};

struct GravSmem {
    int leaf[GW_LEAF];
    int leafoff[GW_LEAF + 1];
    float4 jp[GW_JP];
    float je[GW_JP];
    float4 c0[2][GW_JC], c1[2][GW_JC], c2[2][GW_JC];  // two buffers: one evaluated, one filling
    int4 cnb[GW_JC];  // raw cell corners of the buffer being filled (each thread converts its own slots)
    float4 red[GW_THREADS];
    int ws[32];
    int g;
};

// A cell of `level` must be opened for a group when their boxes overlap or
// when (2 s)^2 > theta^2 d2 in FP64 (s the cell side and d2 the squared
// distance between the cell centre and the group box, both in doubled grid
// units).  That FP64 test is monotone in the integer d2, so the host finds,
// with the same FP64 arithmetic, the largest d2 that passes it for each
// level; the walk then compares integers (no FP64 per visited cell).
__device__ __forceinline__ bool must_open(int4 C, int level, const int *bmin, const int *bmax,
                                          const long long *d2max)
{
    long long s = 1ll << (GNB_MAXLEV - level);
    bool overlap = true;
    long long d2 = 0;
    int cc[3] = {C.x, C.y, C.z};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        long long lo = cc[a], b0 = bmin[a], b1 = bmax[a];
        if (b0 > lo + s - 1 || b1 < lo) overlap = false;
        long long cen = 2 * lo + s;
        long long d = 0;
        if (2 * b0 > cen) d = 2 * b0 - cen;
        else if (cen > 2 * b1) d = cen - 2 * b1;
        d2 += d * d;
    }
    return overlap || d2 <= d2max[level];
}

// FP32 1/sqrt(x) of a squared distance plus softening (a positive normal
// number when no softening is zero): the hardware approximation with
// denormals flushed, a single instruction (relative error below 2^-22).
__device__ __forceinline__ float rsqrt_pos(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Particle-particle: with q.w = -m_j (staged negated), accumulate
// -sum m_j (x_j - x_i)/R^3 and -sum m_j/R, with R^2 = |x_j - x_i|^2 + eps_i^2
// + eps_j^2.  Every sum is accumulated negated (the cell terms below need no
// sign flips that way) and negated once at the end.  MASK (some softening is
// zero): a pair at R = 0 (the particle itself) contributes nothing.
template <bool MASK>
__device__ __forceinline__ void pp_one(float4 q, float e, float xi, float yi, float zi, float e2i, float &ax,
                                       float &ay, float &az, float &ph)
{
    float dx = q.x - xi, dy = q.y - yi, dz = q.z - zi;
    float r2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmaf_rn(dz, dz, e + e2i)));
    float ri;
    if (MASK) ri = r2 > 0.f ? rsqrtf(r2) : 0.f;
    else ri = rsqrt_pos(r2);
    float mr = q.w * ri;
    float mr3 = mr * ri * ri;
    ax = __fmaf_rn(mr3, dx, ax);
    ay = __fmaf_rn(mr3, dy, ay);
    az = __fmaf_rn(mr3, dz, az);
    ph += mr;
}

template <bool MASK>
__device__ __forceinline__ void pp_loop(const GravSmem &S, int np, int split, int js, float xi, float yi, float zi,
                                        float e2i, float &ax, float &ay, float &az, float &ph)
{
#pragma unroll 4
    for (int j = split; j < np; j += js) pp_one<MASK>(S.jp[j], S.je[j], xi, yi, zi, e2i, ax, ay, az, ph);
}

// NI i-particles per thread: each staged j entry is read from shared memory
// once for all of them.
template <int NI, bool MASK>
__device__ __forceinline__ void pp_loopN(const GravSmem &S, int np, int split, int js, const float4 (&pi)[NI],
                                         float4 (&acc)[NI])
{
    constexpr int UNR = NI >= 4 ? 2 : (NI == 2 ? 2 : 4);
#pragma unroll UNR
    for (int j = split; j < np; j += js) {
        const float4 q = S.jp[j];
        const float e = S.je[j];
#pragma unroll
        for (int k = 0; k < NI; k++)
            pp_one<MASK>(q, e, pi[k].x, pi[k].y, pi[k].z, pi[k].w, acc[k].x, acc[k].y, acc[k].z, acc[k].w);
    }
}

// Particle-cell with monopole (+ traceless quadrupole), r = x_i - com:
//   a   += -M r/R^3 + Q r/R^5 - 5/2 (r.Q.r) r/R^7
//   phi += -M/R - 1/2 r.Q.r/R^5         (accumulated with the sign flipped)
// evaluated as t = M/R^3 + 5/2 (r.Q.r/R^5)/R^2, a += (Q r)/R^5 - t r.  In the
// negated sums, with s = com - x_i = -r and a.w = -M (staged negated):
// Q s = -Q r and s.Q.s = r.Q.r, so  -a += (Q s)/R^5 + (-t) s  and
// -phi' += -M/R - 1/2 s.Q.s/R^5, every product the exact negation of the
// one above (no sign flip costs an instruction).
template <bool QUAD>
__device__ __forceinline__ void pc_one(float4 a, float4 b, float4 d, float xi, float yi, float zi, float e2i,
                                       float &ax, float &ay, float &az, float &ph)
{
    float sx = a.x - xi, sy = a.y - yi, sz = a.z - zi;
    float R2 = __fmaf_rn(sx, sx, __fmaf_rn(sy, sy, __fmaf_rn(sz, sz, e2i + d.z)));
    float Ri = rsqrt_pos(R2);
    float Ri2 = Ri * Ri;
    float Ri3 = Ri * Ri2;
    if (QUAD) {
        float qx = __fmaf_rn(b.x, sx, __fmaf_rn(b.w, sy, d.x * sz));
        float qy = __fmaf_rn(b.w, sx, __fmaf_rn(b.y, sy, d.y * sz));
        float qz = __fmaf_rn(d.x, sx, __fmaf_rn(d.y, sy, b.z * sz));
        float rqr = __fmaf_rn(sx, qx, __fmaf_rn(sy, qy, sz * qz));
        float Ri5 = Ri3 * Ri2;
        float rqr5 = rqr * Ri5;
        float nt = __fmaf_rn(rqr5, -2.5f * Ri2, a.w * Ri3);  // -t
        // two chained FMAs per component (Q s/R^5, then -t s)
        ax = __fmaf_rn(nt, sx, __fmaf_rn(qx, Ri5, ax));
        ay = __fmaf_rn(nt, sy, __fmaf_rn(qy, Ri5, ay));
        az = __fmaf_rn(nt, sz, __fmaf_rn(qz, Ri5, az));
        ph = __fmaf_rn(-0.5f, rqr5, __fmaf_rn(a.w, Ri, ph));
    } else {
        float mR3 = a.w * Ri3;  // -M/R^3
        ax = __fmaf_rn(mR3, sx, ax);
        ay = __fmaf_rn(mR3, sy, ay);
        az = __fmaf_rn(mR3, sz, az);
        ph = __fmaf_rn(a.w, Ri, ph);
    }
}

template <int NI, bool QUAD>
__device__ __forceinline__ void pc_loopN(const GravSmem &S, int buf, int nc, int split, int js, const float4 (&pi)[NI],
                                         float4 (&acc)[NI])
{
    constexpr int UNR = NI >= 2 ? 1 : 2;
#pragma unroll UNR
    for (int c = split; c < nc; c += js) {
        const float4 a = S.c0[buf][c], b = S.c1[buf][c], d = S.c2[buf][c];
#pragma unroll
        for (int k = 0; k < NI; k++)
            pc_one<QUAD>(a, b, d, pi[k].x, pi[k].y, pi[k].z, pi[k].w, acc[k].x, acc[k].y, acc[k].z, acc[k].w);
    }
}

// Packed form for two or more i-particles per thread: the thread's particles
// in pairs, one per lane of a float2, evaluated with the FP32x2 instructions
// of sm_100 and later (fma.rn.f32x2, add.rn.f32x2, mul.rn.f32x2: two FP32
// operations per issued instruction, each lane rounded as the scalar one).
// Without UNI, the same operations as pp_one / pc_one on each lane, so the
// sums are the scalar ones bit for bit; the positions are held negated
// (nx = -x_i), which turns x_j - x_i and com - x_i into one addition.  UNI (every particle has
// the same softening eps > 0): eps_i^2 + eps_j^2 is the constant E2 =
// 2 fl(eps^2) for every pair (the same value the general form adds up), and a
// cell's mass-weighted eps^2 is eps^2, so the pair's softening term is E2
// without an addition.
template <int NP>
struct IPair {
    float2 nx[NP], ny[NP], nz[NP], e2[NP];
};
template <int NP>
struct APair {
    float2 ax[NP], ay[NP], az[NP], ph[NP];
};

__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }

template <bool MASK>
__device__ __forceinline__ float2 rsqrt2(float2 r2)
{
    float2 r;
    if (MASK) {
        r.x = r2.x > 0.f ? rsqrtf(r2.x) : 0.f;
        r.y = r2.y > 0.f ? rsqrtf(r2.y) : 0.f;
    } else {
        r.x = rsqrt_pos(r2.x);
        r.y = rsqrt_pos(r2.y);
    }
    return r;
}

template <bool MASK, bool UNI>
__device__ __forceinline__ void pp_two(float4 q, float e, float2 nx, float2 ny, float2 nz, float2 e2i, float2 E2,
                                       float2 &ax, float2 &ay, float2 &az, float2 &ph)
{
    const float2 dx = __fadd2_rn(bc2(q.x), nx), dy = __fadd2_rn(bc2(q.y), ny), dz = __fadd2_rn(bc2(q.z), nz);
    const float2 es = UNI ? E2 : __fadd2_rn(bc2(e), e2i);
    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, es)));
    const float2 ri = rsqrt2<MASK>(r2);
    const float2 mr = __fmul2_rn(bc2(q.w), ri);
    const float2 mr3 = __fmul2_rn(__fmul2_rn(mr, ri), ri);
    ax = __ffma2_rn(mr3, dx, ax);
    ay = __ffma2_rn(mr3, dy, ay);
    az = __ffma2_rn(mr3, dz, az);
    ph = __fadd2_rn(ph, mr);
}

// pc_one on two lanes (s = com - x_i, a.w = -M, negated sums).
template <bool QUAD, bool UNI>
__device__ __forceinline__ void pc_two(float4 a, float4 b, float4 d, float2 nx, float2 ny, float2 nz, float2 e2i,
                                       float2 E2, float2 &ax, float2 &ay, float2 &az, float2 &ph)
{
    const float2 sx = __fadd2_rn(bc2(a.x), nx), sy = __fadd2_rn(bc2(a.y), ny), sz = __fadd2_rn(bc2(a.z), nz);
    const float2 es = UNI ? E2 : __fadd2_rn(e2i, bc2(d.z));
    const float2 R2 = __ffma2_rn(sx, sx, __ffma2_rn(sy, sy, __ffma2_rn(sz, sz, es)));
    const float2 Ri = rsqrt2<false>(R2);
    const float2 Ri2 = __fmul2_rn(Ri, Ri);
    const float2 Ri3 = __fmul2_rn(Ri, Ri2);
    if (QUAD) {
        const float2 qx = __ffma2_rn(bc2(b.x), sx, __ffma2_rn(bc2(b.w), sy, __fmul2_rn(bc2(d.x), sz)));
        const float2 qy = __ffma2_rn(bc2(b.w), sx, __ffma2_rn(bc2(b.y), sy, __fmul2_rn(bc2(d.y), sz)));
        const float2 qz = __ffma2_rn(bc2(d.x), sx, __ffma2_rn(bc2(d.y), sy, __fmul2_rn(bc2(b.z), sz)));
        const float2 rqr = __ffma2_rn(sx, qx, __ffma2_rn(sy, qy, __fmul2_rn(sz, qz)));
        const float2 Ri5 = __fmul2_rn(Ri3, Ri2);
        const float2 rqr5 = __fmul2_rn(rqr, Ri5);
        const float2 nt = __ffma2_rn(rqr5, __fmul2_rn(bc2(-2.5f), Ri2), __fmul2_rn(bc2(a.w), Ri3));
        ax = __ffma2_rn(nt, sx, __ffma2_rn(qx, Ri5, ax));
        ay = __ffma2_rn(nt, sy, __ffma2_rn(qy, Ri5, ay));
        az = __ffma2_rn(nt, sz, __ffma2_rn(qz, Ri5, az));
        ph = __ffma2_rn(bc2(-0.5f), rqr5, __ffma2_rn(bc2(a.w), Ri, ph));
    } else {
        const float2 mR3 = __fmul2_rn(bc2(a.w), Ri3);
        ax = __ffma2_rn(mR3, sx, ax);
        ay = __ffma2_rn(mR3, sy, ay);
        az = __ffma2_rn(mR3, sz, az);
        ph = __ffma2_rn(bc2(a.w), Ri, ph);
    }
}

template <int NP, bool MASK, bool UNI>
__device__ __forceinline__ void pp_loopP(const GravSmem &S, int np, int split, int js, const IPair<NP> &I,
                                         float2 E2, APair<NP> &A)
{
#pragma unroll 4
    for (int j = split; j < np; j += js) {
        const float4 q = S.jp[j];
        const float e = UNI ? 0.f : S.je[j];
#pragma unroll
        for (int k = 0; k < NP; k++)
            pp_two<MASK, UNI>(q, e, I.nx[k], I.ny[k], I.nz[k], I.e2[k], E2, A.ax[k], A.ay[k], A.az[k], A.ph[k]);
    }
}

template <int NP, bool QUAD, bool UNI>
__device__ __forceinline__ void pc_loopP(const GravSmem &S, int buf, int nc, int split, int js, const IPair<NP> &I,
                                         float2 E2, APair<NP> &A)
{
    for (int c = split; c < nc; c += js) {
        const float4 a = S.c0[buf][c], b = S.c1[buf][c], d = S.c2[buf][c];
#pragma unroll
        for (int k = 0; k < NP; k++)
            pc_two<QUAD, UNI>(a, b, d, I.nx[k], I.ny[k], I.nz[k], I.e2[k], E2, A.ax[k], A.ay[k], A.az[k], A.ph[k]);
    }
}

__device__ __forceinline__ int block_scan_excl(int v, int *ws, int *tot)
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

// Appends the entries of the lanes with flag set to a chunk chain (cur: the
// chain's current chunk, cnt: entries in it).  A full chunk is closed and a
// new one taken from the pool; when the pool is exhausted the chain goes dead
// (cur = -1), the pool counter exceeds its capacity and the host repeats the
// walk with a larger pool.
__device__ __forceinline__ void chain_append(bool flag, int val, int &cur, int &cnt, const GravParams &p, int lane)
{
    const unsigned b = __ballot_sync(0xffffffffu, flag);
    if (!b) return;
    const int n = __popc(b), pre = __popc(b & ((1u << lane) - 1u));
    const bool spill = cnt + n > GL_CH;
    int nxt = -1;
    if (spill) {
        if (lane == 0) {
            if (cur >= 0) {
                nxt = atomicAdd(p.top, 1);
                if (nxt >= p.cap) nxt = -1;
                p.cnext[cur] = nxt;
                p.ccnt[cur] = GL_CH;
            }
        }
        nxt = __shfl_sync(0xffffffffu, nxt, 0);
    }
    const int pos = cnt + pre;
    if (flag) {
        if (pos < GL_CH) {
            if (cur >= 0) p.pool[(size_t)cur * GL_CH + pos] = val;
        } else if (nxt >= 0) {
            p.pool[(size_t)nxt * GL_CH + pos - GL_CH] = val;
        }
    }
    if (spill) { cur = nxt; cnt = cnt + n - GL_CH; }
    else cnt += n;
}

__device__ __forceinline__ int chain_new(const GravParams &p, int lane)
{
    int c = 0;
    if (lane == 0) {
        c = atomicAdd(p.top, 1);
        if (c >= p.cap) c = -1;
    }
    return __shfl_sync(0xffffffffu, c, 0);
}

// Closes a chain: records the last chunk's count and pads its unused slots
// with node 0 (a valid index), so a whole chunk can always be copied.
__device__ __forceinline__ void chain_close(const GravParams &p, int cur, int cnt, int lane)
{
    if (cur < 0) return;
    for (int q = cnt + lane; q < GL_CH; q += 32) p.pool[(size_t)cur * GL_CH + q] = 0;
    if (lane == 0) {
        p.ccnt[cur] = cnt;
        p.cnext[cur] = -1;
    }
}

__device__ __forceinline__ void cp_async16_g(void *smem, const void *g)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit_g() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all_g() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Raw data of up to GW_JC accepted cells (two per thread, node indices in
// idx) into buffer b: corner, centre of mass + mass, quadrupole.
__device__ __forceinline__ void cells_issue(GravSmem &S, const GravParams &p, int b, const int *idx)
{
    for (int h = 0; h < 2; h++) {
        const int s = threadIdx.x + h * GW_THREADS, node = idx[h];
        cp_async16_g(&S.cnb[s], &p.nb[node]);
        cp_async16_g(&S.c0[b][s], &p.mo0[node]);
        cp_async16_g(&S.c1[b][s], &p.mo1[node]);
        cp_async16_g(&S.c2[b][s], &p.mo2[node]);
    }
    cp_async_commit_g();
}

// Centre of mass as an FP32 offset from the group's reference grid cell, and
// the mass negated (the sums are accumulated negated, see pc_one).
__device__ __forceinline__ void cells_convert(GravSmem &S, int b, const int *gref, float unit)
{
    for (int h = 0; h < 2; h++) {
        const int s = threadIdx.x + h * GW_THREADS;
        const int4 C = S.cnb[s];
        const float4 m0 = S.c0[b][s];
        S.c0[b][s] = make_float4(grid_off(C.x, gref[0], m0.x, unit), grid_off(C.y, gref[1], m0.y, unit),
                                 grid_off(C.z, gref[2], m0.z, unit), -m0.w);
    }
}

// Leaf variant of chain_append: the entry is the leaf's first particle and
// lcum receives the leaf's offset in the group's concatenated leaf particles.
__device__ __forceinline__ void chain_append_leaf(bool flag, int first, int count, int &npart, int &cur, int &cnt,
                                                  const GravParams &p, int lane)
{
    const unsigned b = __ballot_sync(0xffffffffu, flag);
    if (!b) return;
    int inc = flag ? count : 0;  // inclusive scan of the counts over the appending lanes
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    const int off = npart + inc - (flag ? count : 0);
    npart += __shfl_sync(0xffffffffu, inc, 31);
    const int n = __popc(b), pre = __popc(b & ((1u << lane) - 1u));
    const bool spill = cnt + n > GL_CH;
    int nxt = -1;
    if (spill) {
        if (lane == 0) {
            if (cur >= 0) {
                nxt = atomicAdd(p.top, 1);
                if (nxt >= p.cap) nxt = -1;
                p.cnext[cur] = nxt;
                p.ccnt[cur] = GL_CH;
            }
        }
        nxt = __shfl_sync(0xffffffffu, nxt, 0);
    }
    const int pos = cnt + pre;
    if (flag) {
        size_t slot = (size_t)-1;
        if (pos < GL_CH) {
            if (cur >= 0) slot = (size_t)cur * GL_CH + pos;
        } else if (nxt >= 0) {
            slot = (size_t)nxt * GL_CH + pos - GL_CH;
        }
        if (slot != (size_t)-1) {
            p.pool[slot] = first;
            p.lcum[slot] = off;
        }
    }
    if (spill) { cur = nxt; cnt = cnt + n - GL_CH; }
    else cnt += n;
}

// Tree walk of one group per warp (see the file comment).
__global__ void __launch_bounds__(GL_WARPS * 32, 5) k_grav_walk(GravParams p)
{
    __shared__ int stack[GL_WARPS][GL_STACK];
    __shared__ long long d2max[GNB_MAXLEV + 1];  // lanes index it by level: shared, not the parameter bank
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int *st = stack[w];
    for (int l = threadIdx.x; l <= GNB_MAXLEV; l += blockDim.x) d2max[l] = p.open_d2max[l];
    __syncthreads();
    const int ngroups = *p.ngroups;
    unsigned long long cnt_pp = 0, cnt_pc = 0;
    for (;;) {
        int gi = 0;
        if (lane == 0) gi = atomicAdd(p.next, 1);
        gi = __shfl_sync(0xffffffffu, gi, 0);
        if (gi >= ngroups) break;
        const int4 ga = __ldg(&p.na[p.groups[gi]]);
        const int gfirst = ga.x, gcount = ga.y;
        // bounding box of the group's particle cells
        int bmin[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, bmax[3] = {-1, -1, -1};
        for (int i = gfirst + lane; i < gfirst + gcount; i += 32) {
            const int cc[3] = {p.cx[i], p.cy[i], p.cz[i]};
#pragma unroll
            for (int a = 0; a < 3; a++) { bmin[a] = min(bmin[a], cc[a]); bmax[a] = max(bmax[a], cc[a]); }
        }
#pragma unroll
        for (int a = 0; a < 3; a++)
            for (int o = 16; o > 0; o >>= 1) {
                bmin[a] = min(bmin[a], __shfl_xor_sync(0xffffffffu, bmin[a], o));
                bmax[a] = max(bmax[a], __shfl_xor_sync(0xffffffffu, bmax[a], o));
            }
        int ccur = chain_new(p, lane), lcur = chain_new(p, lane);
        const int chead = ccur, lhead = lcur;
        int ccnt = 0, lcnt = 0, ncell = 0, npart = 0;
        int sp = 1;
        if (lane == 0) st[0] = 0;
        __syncwarp();
        while (sp > 0) {
            // pop up to 32 nodes, keeping room for their children
            int k = min(32, sp);
            const int room = max(1, (GL_STACK - sp) / 7);
            k = min(k, room);
            const int node = lane < k ? st[sp - k + lane] : -1;
            __syncwarp();
            sp -= k;
            bool is_cell = false, is_leaf = false;
            int nch = 0, child0 = 0, lcount = 0, lfirst = 0;
            if (node >= 0) {
                const int4 a = __ldg(&p.na[node]);
                const int lev = a.w & 255;
                const bool open = node == 0 || must_open(__ldg(&p.nb[node]), lev, bmin, bmax, d2max);
                if (!open) is_cell = true;
                else if ((a.w >> 8) == 0) { is_leaf = true; lcount = a.y; lfirst = a.x; }
                else { nch = a.w >> 8; child0 = a.z; }
            }
            // push children (inclusive scan of the child counts over the warp)
            int inc = nch;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            const int tot = __shfl_sync(0xffffffffu, inc, 31);
            const int base = sp + inc - nch;
            for (int q = 0; q < nch; q++) {
                if (base + q < GL_STACK) st[base + q] = child0 + q;
                else atomicOr(p.status, ST_STACK_OVERFLOW);
            }
            sp = min(sp + tot, GL_STACK);
            __syncwarp();
            chain_append(is_cell, node, ccur, ccnt, p, lane);
            chain_append_leaf(is_leaf, lfirst, lcount, npart, lcur, lcnt, p, lane);
            ncell += __popc(__ballot_sync(0xffffffffu, is_cell));
        }
        chain_close(p, ccur, ccnt, lane);
        chain_close(p, lcur, lcnt, lane);
        if (lane == 0) {
            p.ghead[gi] = make_int4(chead, lhead, npart, 0);
            p.gref[gi] = make_int4((bmin[0] + bmax[0]) >> 1, (bmin[1] + bmax[1]) >> 1, (bmin[2] + bmax[2]) >> 1, 0);
        }
        cnt_pc += (unsigned long long)ncell * gcount;
        cnt_pp += (unsigned long long)npart * gcount;
    }
    if (lane == 0) {
        atomicAdd(&p.counters[0], cnt_pp);
        atomicAdd(&p.counters[1], cnt_pc);
    }
}

// One chunk of up to NI * GW_THREADS i-particles of a group against
// the group's lists, NI i-particles per thread.  j-splits: each of the js
// thread sets holds all icnt i-particles (slot s and s + k ilanes, k < NI)
// and takes every js-th j entry, so a small group keeps the CTA busy; with
// more i-particles per thread each staged j entry is read once for all of
// them and fewer partial sums are left to reduce.
template <int NI, bool MASK, bool QUAD, bool UNI>
__device__ __forceinline__ void eval_chunk(GravSmem &S, const GravParams &p, int first, int icnt, const int4 &gh,
                                           const int *gref, float unit)
{
    const int tid = threadIdx.x;
    const int ilanes = (icnt + NI - 1) / NI;
    const int js = GW_THREADS / ilanes;
    const int islot = tid % ilanes, split = tid / ilanes;
    const bool ivalid = split < js;
    // one i-particle: scalar arithmetic; more: packed pairs (pp_two, pc_two)
    constexpr bool PK = NI >= 2;
    constexpr int NP = PK ? NI / 2 : 1;
    float4 pi[NI], acc[NI];
    IPair<NP> I;
    APair<NP> A;
    const float2 E2 = bc2(p.e2u);
#pragma unroll
    for (int k = 0; k < NI; k++) {
        const int sl = islot + k * ilanes;
        const int ip = first + (sl < icnt ? sl : islot);  // an empty slot repeats the first particle
        const float ep = p.eps[ip];
        pi[k] = make_float4(grid_off(p.cx[ip], gref[0], p.rx[ip], unit), grid_off(p.cy[ip], gref[1], p.ry[ip], unit),
                            grid_off(p.cz[ip], gref[2], p.rz[ip], unit), ep * ep);
        acc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if constexpr (PK) {
#pragma unroll
        for (int h = 0; h < NP; h++) {
            I.nx[h] = make_float2(-pi[2 * h].x, -pi[2 * h + 1].x);
            I.ny[h] = make_float2(-pi[2 * h].y, -pi[2 * h + 1].y);
            I.nz[h] = make_float2(-pi[2 * h].z, -pi[2 * h + 1].z);
            I.e2[h] = make_float2(pi[2 * h].w, pi[2 * h + 1].w);
            A.ax[h] = A.ay[h] = A.az[h] = A.ph[h] = make_float2(0.f, 0.f);
        }
    }
    // accepted cells, one chunk at a time, double buffered: while a chunk is
    // evaluated, cp.async fills the other buffer with the next chunk (whose
    // node indices were loaded one chunk earlier).  The first chunk's copy is
    // issued here and lands while the opened leaves below are evaluated.
    int ch = gh.x, cb = 0;
    int idx[2] = {0, 0}, cnx = -1;
    if (ch >= 0) {
        idx[0] = p.pool[(size_t)ch * GL_CH + tid];
        idx[1] = p.pool[(size_t)ch * GL_CH + tid + GW_THREADS];
        cells_issue(S, p, 0, idx);
        cnx = p.cnext[ch];
        if (cnx >= 0) {
            idx[0] = p.pool[(size_t)cnx * GL_CH + tid];
            idx[1] = p.pool[(size_t)cnx * GL_CH + tid + GW_THREADS];
        }
    }
    // opened leaves, one chunk at a time: each entry holds the leaf's first
    // particle and its offset in the group's leaf particles (from the walk),
    // so particles are staged in batches of GW_JP without a scan or a node
    // lookup
    for (int lch = gh.y; lch >= 0;) {
        const int nl = p.ccnt[lch];
        const int lnx = p.cnext[lch];
        // only a chain's head chunk can be empty (a group with no opened leaf)
        const int base = nl > 0 ? p.lcum[(size_t)lch * GL_CH] : 0;
        const int end = lnx >= 0 ? p.lcum[(size_t)lnx * GL_CH] : gh.z;
        const int total = nl > 0 ? end - base : 0;
        for (int q = tid; q < nl; q += GW_THREADS) {
            S.leaf[q] = p.pool[(size_t)lch * GL_CH + q];
            S.leafoff[q] = p.lcum[(size_t)lch * GL_CH + q] - base;
        }
        if (tid == 0) S.leafoff[nl] = total;
        __syncthreads();
        for (int c0 = 0; c0 < total; c0 += GW_JP) {
            const int np = min(GW_JP, total - c0);
            for (int k = tid; k < np; k += GW_THREADS) {
                const int pos = c0 + k;
                int lo = 0, hi = nl - 1;  // the leaf holding position pos
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (S.leafoff[mid] <= pos) lo = mid;
                    else hi = mid - 1;
                }
                const int j = S.leaf[lo] + (pos - S.leafoff[lo]);
                const float ej = p.eps[j];
                S.jp[k] = make_float4(grid_off(p.cx[j], gref[0], p.rx[j], unit),
                                      grid_off(p.cy[j], gref[1], p.ry[j], unit),
                                      grid_off(p.cz[j], gref[2], p.rz[j], unit), -p.m[j]);
                S.je[k] = ej * ej;
            }
            __syncthreads();
            if (ivalid) {
                if constexpr (PK) pp_loopP<NP, MASK, UNI>(S, np, split, js, I, E2, A);
                else pp_loopN<NI, MASK>(S, np, split, js, pi, acc);
            }
            __syncthreads();
        }
        lch = lnx;
    }
    if (ch >= 0) {
        cp_async_wait_all_g();
        cells_convert(S, 0, gref, unit);
        __syncthreads();
    }
    while (ch >= 0) {
        const int nc = p.ccnt[ch];
        int nxt2 = -1, idx2[2] = {0, 0};
        if (cnx >= 0) {
            cells_issue(S, p, cb ^ 1, idx);
            nxt2 = p.cnext[cnx];
            if (nxt2 >= 0) {
                idx2[0] = p.pool[(size_t)nxt2 * GL_CH + tid];
                idx2[1] = p.pool[(size_t)nxt2 * GL_CH + tid + GW_THREADS];
            }
        }
        if (ivalid) {
            if constexpr (PK) pc_loopP<NP, QUAD, UNI>(S, cb, nc, split, js, I, E2, A);
            else pc_loopN<NI, QUAD>(S, cb, nc, split, js, pi, acc);
        }
        if (cnx >= 0) {
            cp_async_wait_all_g();
            cells_convert(S, cb ^ 1, gref, unit);
        }
        __syncthreads();  // buffer cb evaluated by all; buffer cb ^ 1 converted by all
        ch = cnx;
        cnx = nxt2;
        idx[0] = idx2[0];
        idx[1] = idx2[1];
        cb ^= 1;
    }
    // reduce the j-splits: the partial sums of particle slots k0 .. k0 + RB - 1
    // at a time go through the PP staging buffer (idle here)
    constexpr int RB = GW_JP / GW_THREADS;
    // the sums were accumulated negated
    if constexpr (PK) {
#pragma unroll
        for (int h = 0; h < NP; h++) {
            acc[2 * h] = make_float4(-A.ax[h].x, -A.ay[h].x, -A.az[h].x, -A.ph[h].x);
            acc[2 * h + 1] = make_float4(-A.ax[h].y, -A.ay[h].y, -A.az[h].y, -A.ph[h].y);
        }
    } else {
#pragma unroll
        for (int k = 0; k < NI; k++) acc[k] = make_float4(-acc[k].x, -acc[k].y, -acc[k].z, -acc[k].w);
    }
#pragma unroll
    for (int k0 = 0; k0 < NI; k0 += RB) {
#pragma unroll
        for (int k = k0; k < NI && k < k0 + RB; k++) S.jp[(k - k0) * GW_THREADS + tid] = acc[k];
        __syncthreads();
        if (split == 0 && ivalid) {
#pragma unroll
            for (int k = k0; k < NI && k < k0 + RB; k++) {
                const int sl = islot + k * ilanes;
                if (sl >= icnt) continue;
                float4 a = acc[k];
                for (int s2 = 1; s2 < js; s2++) {
                    const float4 r = S.jp[(k - k0) * GW_THREADS + tid + s2 * ilanes];
                    a.x += r.x; a.y += r.y; a.z += r.z; a.w += r.w;
                }
                const int ip = first + sl;
                if (!MASK) {  // remove the j == i term (eps reloaded: no register holds it through the loops)
                    const float ep = p.eps[ip];
                    a.w -= p.m[ip] * rsqrtf(2.f * (ep * ep));
                }
                p.ax[ip] = p.G * a.x;
                p.ay[ip] = p.G * a.y;
                p.az[ip] = p.G * a.z;
                p.pot[ip] = -p.G * a.w;
            }
        }
        __syncthreads();
    }
}

// Evaluation of the walk's lists, one group per CTA (see the file comment):
// the group's particles in chunks of up to NIMAX * GW_THREADS, eight per
// thread above 128 particles in a chunk (NIMAX = 8), four above 64, two above
// 16, else one.  Five CTAs per SM (96 registers a thread; the eight-particle
// variant spills a few bytes outside its inner loops and still runs faster
// than at 4 CTAs and 128 registers).
template <bool MASK, bool QUAD, int NIMAX, bool UNI>
__global__ void __launch_bounds__(GW_THREADS, 5) k_grav_eval(GravParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GravSmem &S = *reinterpret_cast<GravSmem *>(smem_raw);
    const int tid = threadIdx.x;
    const float unit = (float)p.box[4];
    const int ngroups = *p.ngroups;
    for (;;) {
        if (tid == 0) S.g = atomicAdd(p.next, 1);
        __syncthreads();
        const int gi = S.g;
        if (gi >= ngroups) break;
        const int4 ga = p.na[p.groups[gi]];
        const int gfirst = ga.x, gcount = ga.y;
        const int4 gh = p.ghead[gi];
        const int4 gr = p.gref[gi];
        const int gref[3] = {gr.x, gr.y, gr.z};
        for (int i0 = 0; i0 < gcount; i0 += NIMAX * GW_THREADS) {
            const int icnt = min(NIMAX * GW_THREADS, gcount - i0);
            if (NIMAX >= 8 && icnt > 128)
                eval_chunk<NIMAX >= 8 ? 8 : 4, MASK, QUAD, UNI>(S, p, gfirst + i0, icnt, gh, gref, unit);
            else if (icnt > 64) eval_chunk<4, MASK, QUAD, UNI>(S, p, gfirst + i0, icnt, gh, gref, unit);
            else if (icnt > 16) eval_chunk<2, MASK, QUAD, UNI>(S, p, gfirst + i0, icnt, gh, gref, unit);
            else eval_chunk<1, MASK, QUAD, UNI>(S, p, gfirst + i0, icnt, gh, gref, unit);
        }
    }
}

// Direct summation: every group streams all n particles through shared memory.
template <bool MASK>
__global__ void __launch_bounds__(GW_THREADS, 4) k_gravity_direct(GravParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GravSmem &S = *reinterpret_cast<GravSmem *>(smem_raw);
    const int tid = threadIdx.x;
    const float unit = (float)p.box[4];
    const int ngroups = *p.ngroups;
    for (;;) {
        if (tid == 0) S.g = atomicAdd(p.next, 1);
        __syncthreads();
        const int gi = S.g;
        if (gi >= ngroups) break;
        const int4 ga = p.na[p.groups[gi]];
        for (int i0 = 0; i0 < ga.y; i0 += GW_THREADS) {
            const int icnt = min(GW_THREADS, ga.y - i0);
            const int ilanes = icnt;
            const int js = GW_THREADS / ilanes;
            const int islot = tid % ilanes, split = tid / ilanes;
            const bool ivalid = split < js;
            const int ip = ga.x + i0 + islot;
            const int gref[3] = {p.cx[ga.x + i0], p.cy[ga.x + i0], p.cz[ga.x + i0]};
            const float xi = grid_off(p.cx[ip], gref[0], p.rx[ip], unit);
            const float yi = grid_off(p.cy[ip], gref[1], p.ry[ip], unit);
            const float zi = grid_off(p.cz[ip], gref[2], p.rz[ip], unit);
            const float e2i = p.eps[ip] * p.eps[ip];
            float ax = 0.f, ay = 0.f, az = 0.f, ph = 0.f;
            for (int c0 = 0; c0 < p.n; c0 += GW_JP) {
                int np = min(GW_JP, p.n - c0);
                __syncthreads();
                for (int k = tid; k < np; k += GW_THREADS) {
                    int j = c0 + k;
                    float ej = p.eps[j];
                    S.jp[k] = make_float4(grid_off(p.cx[j], gref[0], p.rx[j], unit),
                                          grid_off(p.cy[j], gref[1], p.ry[j], unit),
                                          grid_off(p.cz[j], gref[2], p.rz[j], unit), -p.m[j]);
                    S.je[k] = ej * ej;
                }
                __syncthreads();
                if (ivalid) pp_loop<MASK>(S, np, split, js, xi, yi, zi, e2i, ax, ay, az, ph);
            }
            __syncthreads();
            ax = -ax; ay = -ay; az = -az; ph = -ph;  // the sums were accumulated negated
            S.red[tid] = make_float4(ax, ay, az, ph);
            __syncthreads();
            if (split == 0 && ivalid) {
                for (int s2 = 1; s2 < js; s2++) {
                    float4 r = S.red[tid + s2 * ilanes];
                    ax += r.x; ay += r.y; az += r.z; ph += r.w;
                }
                if (!MASK) ph -= p.m[ip] * rsqrtf(2.f * e2i);
                p.ax[ip] = p.G * ax;
                p.ay[ip] = p.G * ay;
                p.az[ip] = p.G * az;
                p.pot[ip] = -p.G * ph;
            }
        }
        __syncthreads();
    }
}

static int g_sms = 0;

static GravParams make_params(gnb_ctx *c)
{
    PArr &a = c->P[c->cur];
    GravParams p;
    p.na = c->t.na; p.nb = c->t.nb; p.mo0 = c->t.mo0; p.mo1 = c->t.mo1; p.mo2 = c->t.mo2;
    p.groups = c->t.groups; p.ngroups = c->t.ngroups_d;
    p.cx = a.cx; p.cy = a.cy; p.cz = a.cz; p.rx = a.rx; p.ry = a.ry; p.rz = a.rz;
    p.m = a.m; p.eps = a.eps;
    p.ax = c->gax; p.ay = c->gay; p.az = c->gaz; p.pot = c->pot;
    p.box = c->box_d;
    p.theta2 = c->cfg.theta * c->cfg.theta;
    for (int l = 0; l <= GNB_MAXLEV; l++) {
        // largest d2 with (2 s)^2 > theta2 * (double)d2 (the test is monotone
        // in d2; (double)d2 rounds the same way here and on the device)
        const long long sz = 1ll << (GNB_MAXLEV - l);
        const double lhs = (double)(2 * sz) * (double)(2 * sz);
        long long lo = 0, hi = (1ll << 62);
        if (!(lhs > p.theta2 * (double)hi)) {
            while (hi - lo > 1) {  // invariant: lo passes, hi fails
                const long long mid = lo + (hi - lo) / 2;
                if (lhs > p.theta2 * (double)mid) lo = mid;
                else hi = mid;
            }
            p.open_d2max[l] = lo;
        } else {
            p.open_d2max[l] = hi;  // theta = 0: every cell opens
        }
    }
    p.G = (float)c->cfg.G;
    p.e2u = c->eps_uniform ? 2.f * (c->eps0 * c->eps0) : 0.f;
    p.quad = c->cfg.multipole;
    p.n = (int)c->n;
    p.next = c->pinned_i ? nullptr : nullptr;
    p.status = c->status_d;
    p.counters = c->counters_d;
    return p;
}

template <class K>
static int launch_persistent(gnb_ctx *c, K kern, GravParams p, int *next_d)
{
    size_t smem = sizeof(GravSmem);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(c, e, "gravity smem attribute");
    if (g_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, GW_THREADS, smem);
    if (per_sm < 1) per_sm = 1;
    p.next = next_d;
    cudaMemsetAsync(next_d, 0, sizeof(int), c->s);
    gnb::counted(kern)<<<g_sms * per_sm, GW_THREADS, smem, c->s>>>(p);
    GNB_LAUNCH_CHECK(c, "gravity kernel");
    return GNB_OK;
}

// Interaction-list pool: group arrays for the current tree, chunks for `chunks`.
// The group count itself stays on the device (reading it would synchronise);
// the tree's node count, known on the host after every build, bounds it.
static int lists_alloc(gnb_ctx *c, int chunks)
{
    const int ng = std::max(c->t.nnodes, 1);
    if (c->gl_gcap < ng) {
        dfree(c, c->gl_head); dfree(c, c->gl_ref);
        c->gl_head = nullptr; c->gl_ref = nullptr;
        const int cap = ng + ng / 4 + 64;
        GNB_TRY(dalloc(c, &c->gl_head, (size_t)cap));
        GNB_TRY(dalloc(c, &c->gl_ref, (size_t)cap));
        c->gl_gcap = cap;
    }
    if (c->gl_cap < chunks) {
        // grow geometrically with headroom: the estimate follows the node
        // count, which drifts from step to step, and a reallocation (cudaFree
        // synchronises the device) must not recur every step
        chunks = std::max(chunks + chunks / 4, c->gl_cap + c->gl_cap / 2);
        dfree(c, c->gl_pool); dfree(c, c->gl_next); dfree(c, c->gl_cnt); dfree(c, c->gl_lcum);
        c->gl_pool = nullptr; c->gl_next = nullptr; c->gl_cnt = nullptr; c->gl_lcum = nullptr;
        GNB_TRY(dalloc(c, &c->gl_pool, (size_t)chunks * GL_CH));
        GNB_TRY(dalloc(c, &c->gl_lcum, (size_t)chunks * GL_CH));
        GNB_TRY(dalloc(c, &c->gl_next, (size_t)chunks));
        GNB_TRY(dalloc(c, &c->gl_cnt, (size_t)chunks));
        c->gl_cap = chunks;
    }
    if (!c->gl_top) GNB_TRY(dalloc(c, &c->gl_top, 1));
    return GNB_OK;
}

int gravity_tree(gnb_ctx *c)
{
    // first guess: two chunks per possible group (cells, leaves) plus 16 list
    // entries per particle
    const int want = 2 * c->t.nnodes + (int)((16 * (long long)c->n) / GL_CH) + 1024;
    GNB_TRY(lists_alloc(c, std::max(c->gl_cap, want)));
    int *next_d = (int *)(c->counters_d + 6);
    for (int attempt = 0;; attempt++) {
        GravParams p = make_params(c);
        p.pool = c->gl_pool; p.cnext = c->gl_next; p.ccnt = c->gl_cnt; p.top = c->gl_top; p.lcum = c->gl_lcum;
        p.ghead = c->gl_head; p.gref = c->gl_ref; p.cap = c->gl_cap;
        p.next = next_d;
        cudaMemsetAsync(c->counters_d, 0, 2 * sizeof(unsigned long long), c->s);
        cudaMemsetAsync(c->gl_top, 0, sizeof(int), c->s);
        cudaMemsetAsync(next_d, 0, sizeof(int), c->s);
        if (g_sms == 0) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        }
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grav_walk, GL_WARPS * 32, 0);
        gnb::counted(k_grav_walk)<<<g_sms * std::max(per_sm, 1), GL_WARPS * 32, 0, c->s>>>(p);
        GNB_LAUNCH_CHECK(c, "tree walk");
        // the pool must have held every list; otherwise grow it and walk again
        GNB_TRY(cuda_check(c, cudaMemcpyAsync(&c->pinned_i[40], c->gl_top, sizeof(int), cudaMemcpyDeviceToHost, c->s),
                           "list pool read"));
        GNB_TRY(cuda_check(c, cudaStreamSynchronize(c->s), "list pool sync"));
        const int used = c->pinned_i[40];
        if (used <= c->gl_cap) {
            const bool q = c->cfg.multipole != 0;
            // groups of more than 128 particles: eight i-particles per thread
            if (c->cfg.n_group > 128) {
                if (c->min_eps_zero) {
                    if (q) return launch_persistent(c, k_grav_eval<true, true, 8, false>, p, next_d);
                    return launch_persistent(c, k_grav_eval<true, false, 8, false>, p, next_d);
                }
                if (c->eps_uniform) {
                    if (q) return launch_persistent(c, k_grav_eval<false, true, 8, true>, p, next_d);
                    return launch_persistent(c, k_grav_eval<false, false, 8, true>, p, next_d);
                }
                if (q) return launch_persistent(c, k_grav_eval<false, true, 8, false>, p, next_d);
                return launch_persistent(c, k_grav_eval<false, false, 8, false>, p, next_d);
            }
            if (c->min_eps_zero) {
                if (q) return launch_persistent(c, k_grav_eval<true, true, 4, false>, p, next_d);
                return launch_persistent(c, k_grav_eval<true, false, 4, false>, p, next_d);
            }
            if (c->eps_uniform) {
                if (q) return launch_persistent(c, k_grav_eval<false, true, 4, true>, p, next_d);
                return launch_persistent(c, k_grav_eval<false, false, 4, true>, p, next_d);
            }
            if (q) return launch_persistent(c, k_grav_eval<false, true, 4, false>, p, next_d);
            return launch_persistent(c, k_grav_eval<false, false, 4, false>, p, next_d);
        }
        if (attempt >= 4) return fail(c, GNB_ECAPACITY, "interaction-list pool");
        GNB_TRY(lists_alloc(c, used + used / 2 + 1024));
    }
}

int gravity_direct(gnb_ctx *c)
{
    GravParams p = make_params(c);
    int *next_d = (int *)(c->counters_d + 6);
    if (c->min_eps_zero) return launch_persistent(c, k_gravity_direct<true>, p, next_d);
    return launch_persistent(c, k_gravity_direct<false>, p, next_d);
}

// ---------------------------------------------------------------- NFW halo
// M(<r) = Ms [ln(1+r/rs) - (r/rs)/(1+r/rs)], a = -G M(<r) x / r^3,
// Phi = -G Ms ln(1 + r/rs) / r.
//
// The bracket cancels for small s = r/rs (both terms ~ s, the difference
// ~ s^2/2), which in FP32 would cost ~ 2^-24 / s of relative accuracy.  With
// t = s/(1+s), ln(1+s) = -ln(1-t) = sum_k t^k/k, so the bracket is
// sum_{k>=2} t^k / k, a series of positive terms; below s = 1/4 (t = 1/5)
// its first 11 terms leave a relative truncation error below 2e-8, and above
// it the direct form loses at most a factor 10 (< 1e-6).
__device__ __forceinline__ float nfw_bracket(float s)
{
    if (s >= 0.25f) return log1pf(s) - s / (1.f + s);
    const float t = s / (1.f + s);
    float sum = 1.f / 12.f;  // Horner in t over 1/2 + t/3 + ... + t^10/12
    for (int k = 11; k >= 2; k--) sum = __fmaf_rn(sum, t, 1.f / (float)k);
    return t * t * sum;
}

__global__ void k_nfw(const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
                      int n, float G, float ms, float rs, float *__restrict__ ax, float *__restrict__ ay,
                      float *__restrict__ az, float *__restrict__ pext)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float px = (float)x[i], py = (float)y[i], pz = (float)z[i];
    float r = sqrtf(px * px + py * py + pz * pz);
    float s = r / rs;
    float l1 = log1pf(s);
    float menc = ms * nfw_bracket(s);
    float f = r > 0.f ? -G * menc / (r * r * r) : 0.f;
    ax[i] = f * px;
    ay[i] = f * py;
    az[i] = f * pz;
    pext[i] = r > 0.f ? -G * ms * l1 / r : -G * ms / rs;
}

int gravity_nfw(gnb_ctx *c)
{
    int n = (int)c->n;
    PArr &a = c->P[c->cur];
    if (c->cfg.nfw_ms > 0) {
        gnb::counted(k_nfw)<<<(n + 255) / 256, 256, 0, c->s>>>(a.x, a.y, a.z, n, (float)c->cfg.G, (float)c->cfg.nfw_ms,
                                                 (float)c->cfg.nfw_rs, c->ax, c->ay, c->az, c->pext);
        GNB_LAUNCH_CHECK(c, "nfw");
    } else {
        cudaMemsetAsync(c->ax, 0, sizeof(float) * n, c->s);
        cudaMemsetAsync(c->ay, 0, sizeof(float) * n, c->s);
        cudaMemsetAsync(c->az, 0, sizeof(float) * n, c->s);
        cudaMemsetAsync(c->pext, 0, sizeof(float) * n, c->s);
    }
    return GNB_OK;
}

}  // namespace gnb
