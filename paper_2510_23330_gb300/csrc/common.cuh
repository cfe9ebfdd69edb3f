// common.cuh -- internal declarations of the GB300 N-body/SPH library.
//
// Device data layout (all arrays live in HBM, structure of arrays, particles
// in Morton order after every tree build):
//   x, y, z      double   master positions (Sec. 4.3: FP64 storage)
//   cx, cy, cz   int32    Morton grid cell of the particle (21 bits per axis)
//   rx, ry, rz   float    residual x - (lo + c*unit), in [0, unit)
//   vx, vy, vz   float    velocity; m, eps, u float; type uint8; id int64
//   orig         int32    index of the particle in the caller's arrays
//   grank        int32    rank among gas particles in the caller's order
// Pair arithmetic uses the exact integer cell difference plus the FP32
// residual difference, so an FP32 offset between any two particles carries
// one rounding (relative 2^-24) without FP64 arithmetic.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <utility>
#include <vector>

#include "../../include/galnb.h"

#define GNB_MAXLEV 21
#define GNB_GRID_MAX 2097151

namespace gnb {

// Kernel launches issued by this library (every launch goes through counted()).
extern std::atomic<long long> g_launches;
template <class K>
inline K counted(K k)
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return k;
}

// Device-side status word bits (set by kernels, read by the host).
enum : int {
    ST_TREE_OVERFLOW = 1,
    ST_STACK_OVERFLOW = 2,
    ST_KNN_OVERFLOW = 4,
    ST_SYM_OVERFLOW = 8,
    ST_BAD_INPUT = 16,
};

struct Tree {
    int cap = 0;       // node capacity
    int nnodes = 0;    // nodes of the last build (host copy)
    int depth = GNB_MAXLEV;  // deepest non-empty level of the last build (host copy)
    // node arrays
    int4 *na = nullptr;   // {first, count, child, (nchild << 8) | level}
    int4 *nb = nullptr;   // {corner x, corner y, corner z, parent}
    float4 *mo0 = nullptr; // {com_off x, y, z (rel. to corner, physical), M}
    float4 *mo1 = nullptr; // {Qxx, Qyy, Qzz, Qxy}
    float4 *mo2 = nullptr; // {Qxz, Qyz, eps2, 0}
    int *lvl = nullptr;    // device: level begin offsets [GNB_MAXLEV + 2]
    int *head = nullptr;   // build: the parent of a first child, else -1 [cap]
    // build scratch, per sorted slot and per tile of slots
    int *span = nullptr;   // nodes starting at each slot: first and last level, group level
    int *tcnt = nullptr;   // nodes of each level (and groups) per tile, then their offsets
    int *tot = nullptr;    // nodes of each level (and groups) in all
    int scap = 0, tcap = 0;
    int *groups = nullptr; // group node ids, ascending first particle
    int *ngroups_d = nullptr;
    int ngroups = 0;
};

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace gnb

namespace gnb {
// Per-particle arrays that move with the particle when the set is re-sorted.
struct PArr {
    double *x = nullptr, *y = nullptr, *z = nullptr, *h2 = nullptr;
    int64_t *id = nullptr;
    float *vx = nullptr, *vy = nullptr, *vz = nullptr, *m = nullptr, *eps = nullptr, *u = nullptr;
    float *rx = nullptr, *ry = nullptr, *rz = nullptr;
    float *vpx = nullptr, *vpy = nullptr, *vpz = nullptr, *up = nullptr;  // predicted v, u
    int *orig = nullptr, *grank = nullptr, *cx = nullptr, *cy = nullptr, *cz = nullptr;
    uint8_t *type = nullptr;
};
}  // namespace gnb

struct gnb_ctx {
    gnb_config cfg;
    cudaStream_t s = nullptr;
    std::string err;
    int64_t n = 0, n_gas = 0;
    int64_t cap = 0;          // particle capacity
    bool min_eps_zero = false;
    bool eps_uniform = false;  // every particle has the softening eps0 > 0
    bool slots_caller = false; // the slots still hold the caller's order (no sort since the upload)
    float knn_margin = 1.05f;   // kernel-size search radius over the previous support (adapted per evaluation)
    float eps0 = 0.f;

    gnb::PArr P[2];
    int cur = 0;              // P[cur] holds the particles
    // per-slot results of the last force evaluation (not permuted)
    float *ax = nullptr, *ay = nullptr, *az = nullptr, *pot = nullptr, *dudt = nullptr;
    float *gax = nullptr, *gay = nullptr, *gaz = nullptr;  // self-gravity part
    float *pext = nullptr;                                  // external potential
    float *rho = nullptr, *pres = nullptr, *cs = nullptr;   // gas fields per slot
    // sort scratch
    uint64_t *skey = nullptr, *skey2 = nullptr;
    float *kres = nullptr;    // remainders of the coordinates within their grid cells [3][cap], slot order
    int *sval = nullptr, *sval2 = nullptr, *slot_of_orig = nullptr, *src = nullptr;
    int *pscan = nullptr;     // per-slot scan scratch
    unsigned char *tmp_out = nullptr;  // export staging (8 bytes per particle)
    int *rs_counts = nullptr, *rs_total = nullptr;
    int rs_tiles_cap = 0;
    // root box: device {lo[3], L, unit} plus min/max scratch
    double *box_d = nullptr;
    unsigned long long *mm_d = nullptr;
    double lo[3] = {0, 0, 0}, L = 1, unit = 1;
    // gravity tree
    gnb::Tree t;
    // hydro (gas) arrays, gas order = Morton order of the gas particles
    int64_t gcap = 0;
    int *gslot = nullptr;         // particle slot of each gas particle
    int *gas_flag = nullptr, *ngas_d = nullptr;
    uint64_t *gkey = nullptr;
    gnb::Tree gt;                 // hydro tree over gas
    int *gcx = nullptr, *gcy = nullptr, *gcz = nullptr, *ggrank = nullptr;
    float *grx = nullptr, *gry = nullptr, *grz = nullptr;
    double *gx = nullptr, *gy = nullptr, *gz = nullptr;
    float *gm = nullptr, *gvx = nullptr, *gvy = nullptr, *gvz = nullptr, *gu = nullptr;
    double *gh2 = nullptr;        // exact FP64 d^2 of the n_ngb-th neighbour
    float *gh = nullptr;          // h in FP32
    int *g64 = nullptr;           // gas rank of the n_ngb-th neighbour
    float *grho = nullptr, *gP = nullptr, *gcs = nullptr;
    float *gRprev = nullptr;      // search radius hint per gas particle
    float *gE = nullptr;          // FP32 distance error bound used for the particle's list
    float *gvsig = nullptr;       // largest pair signal velocity of the last force pass
    unsigned long long *mut = nullptr;  // per gas particle: mutual-neighbour bits
    int *nbr = nullptr;           // n_gas * 64 gas indices
    float *nd2 = nullptr;         // n_gas * 64 FP32 d^2
    int *rcnt = nullptr, *roff = nullptr, *rfill = nullptr, *rlist = nullptr;
    int *rtot_d = nullptr;
    int64_t rlist_cap = 0;
    float *hax = nullptr, *hay = nullptr, *haz = nullptr, *hdu = nullptr;
    int *kflag = nullptr;         // per hydro group: needs another pass
    float *kR = nullptr;          // per hydro group search radius
    float2 *kRb = nullptr;        // per hydro group radius bracket (too small, too large)
    int2 *kitem = nullptr;        // kNN work items (first, count); groups then split particles
    int *kwl[2] = {nullptr, nullptr};  // kNN worklists: items a pass hands to the next (ping-pong)
    float *gh2lo = nullptr, *gh2hi = nullptr;  // h^2 rounded down / up to FP32 (per gas)
    // per-gas records the hydro force gathers for neighbour j (one pass packs them)
    int4 *fC = nullptr;           // cell x, y, z, mass bits
    float4 *fR = nullptr;         // residual x, y, z, 1/h
    float4 *fV = nullptr;         // v x, y, z, sound speed
    float4 *fQ = nullptr;         // rho, Y, U, - (pair coefficient U_j Y_i of gW(h_i); see sph.cu)
    int *kcount_d = nullptr;

    // supernova surrogate (surrogate.cu)
    int *sreg = nullptr;          // region of each particle slot (-1: none)
    int *rcount = nullptr;        // members per region
    float *vacc = nullptr;        // voxel accumulators: [voxels][4], then [voxels / 2][4] (see k_vox_scatter)
    float *vout = nullptr;        // standardised channels [nreg][grid^3][5]
    double *vw = nullptr;         // remap weights [nreg][grid^3]
    double *vcdf = nullptr;       // remap line CDFs [nreg][axis][grid^2 lines][grid]
    float *vcdf32 = nullptr;      // the same, rounded to FP32 (decides the comparisons it can)
    float *vcdfc = nullptr;       // every 8th FP32 sum of each line (its last entry = the line total)
    double *cent_d = nullptr;     // region centres [nreg][3]
    float *rsx = nullptr;         // region centre x (FP32), sorted ascending (membership search)
    int *rsi = nullptr;           // region index of each sorted entry
    float *centf = nullptr;       // FP32 copy of the centres (membership pre-filter)
    std::vector<int> rs_order;    // host staging of rsi / rsx / centf
    std::vector<float> rs_x, rs_cf;
    float4 *vpa = nullptr, *vpb = nullptr, *vpc = nullptr;  // voxelisation: staged FP32 values per particle
    int *vbox = nullptr;          // voxelisation: packed x and y footprint ranges per particle
    int64_t sur_pcap = 0;         // particle capacity of sreg and the staged arrays
    uint64_t sur_gen = 0;         // bumped whenever a surrogate buffer is reallocated
    unsigned long long *seed_d = nullptr;
    size_t sur_nv = 0;
    int sur_nreg = 0;
    cudaGraphExec_t sn_graph = nullptr;  // captured voxelise -> U-Net -> remap
    // pipelined batch: the U-Net and the remap of region chunks run on their
    // own streams, chunk k's stages ordered by events
    static constexpr int SN_MAXCH = 16;
    cudaStream_t sn_st[2] = {nullptr, nullptr};
    cudaEvent_t sn_ev[3][SN_MAXCH] = {};
    int sn_chunks = 1;                // region chunks of the pipelined batch (1: stages in sequence)
    // asynchronous surrogate batch (submitted now, applied later): a snapshot
    // of the region members (state, caller index, ID, region), worked on a
    // side stream; sna_inv maps caller index -> current slot at apply time
    bool sna_pending = false;
    int sna_nreg = 0, sna_grid = 0, sna_sweeps = 0;
    double sna_side = 0.0;
    void *sna_net = nullptr;
    int64_t sna_cap = 0;
    double *sna_x = nullptr, *sna_y = nullptr, *sna_z = nullptr, *sna_h2 = nullptr;
    float *sna_m = nullptr, *sna_u = nullptr, *sna_vx = nullptr, *sna_vy = nullptr, *sna_vz = nullptr;
    float *sna_rho = nullptr;
    int *sna_reg = nullptr, *sna_orig = nullptr, *sna_pos = nullptr, *sna_inv = nullptr;
    int64_t *sna_id = nullptr;
    unsigned long long *sna_seed = nullptr;
    float *sna_yout = nullptr;    // the network's predictions of the pending batch
    cudaStream_t sna_st = nullptr;
    cudaEvent_t sna_ev_snap = nullptr, sna_ev_done = nullptr;
    int sn_key[4] = {0, 0, 0, 0};
    void *sn_net = nullptr;
    double sn_side = 0.0;
    int64_t sn_n = 0;
    int sn_cur = -1;
    uint64_t sn_gen = 0;          // sur_gen when the graph was captured
    int64_t sn_graph_replays = 0;

    // status / counters
    int *status_d = nullptr;
    int *n_d = nullptr;                        // device copy of n
    unsigned long long *counters_d = nullptr;  // [8]
    int *work_d = nullptr;                     // work counters of persistent kernels [8]
    int *scan_part = nullptr, *scan_poff = nullptr;  // device_scan scratch [1100]
    // tree-gravity interaction lists (gravity.cu): chunk pool and per-group heads
    int *gl_pool = nullptr, *gl_next = nullptr, *gl_cnt = nullptr, *gl_top = nullptr, *gl_lcum = nullptr;
    int4 *gl_head = nullptr, *gl_ref = nullptr;
    int gl_cap = 0, gl_gcap = 0;
    int *pinned_i = nullptr;                   // pinned host scratch [64]
    // hierarchical timesteps (integrate.cu): per particle slot, permuted with
    // the particles by every sort while hier_on; [2] = current and scratch
    bool hier_on = false, hier_valid = false;
    int64_t hier_cap = 0;
    long long *hT0[2] = {nullptr, nullptr}, *hT1[2] = {nullptr, nullptr};  // step start, end (ticks)
    int *hlev[2] = {nullptr, nullptr};
    float4 *hacc[2] = {nullptr, nullptr};  // a_x, a_y, a_z, du/dt of the particle's last update
    int *hkc = nullptr;                    // CFL level per slot (gas) of the last force pass
    unsigned long long *hred = nullptr;    // {next tick (min), updates, wake-ups, status}
    unsigned long long *hred_h = nullptr;  // pinned copy
    double *red_d = nullptr;                   // reduction scratch
    int64_t stats[GNB_S_COUNT_] = {0};
    // replacement by ID (replace.cu): the held IDs sorted with their caller
    // indices (built on the first replacement after gnb_set_particles), and
    // per-call staging of the incoming particles
    bool rid_valid = false;
    int64_t rid_cap = 0, rep_cap = 0, rep_scap = 0;
    uint64_t *rid_key = nullptr, *rid_key2 = nullptr;
    int *rid_orig = nullptr, *rid_orig2 = nullptr, *rid_inv = nullptr, *rid_mark = nullptr;
    unsigned char *rep_buf = nullptr;   // incoming id, x, y, z, vx, vy, vz, u (48 B per particle)
    int *rep_slot = nullptr;            // slot of each incoming particle

    // per-phase CUDA-event timers (enabled by gnb_set_timing)
    bool timing = false;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pend;
    std::vector<cudaEvent_t> evpool;
    double phase_ms[GNB_T_COUNT_] = {0};
    int64_t phase_calls[GNB_T_COUNT_] = {0};
    long long launch_base = 0;
    cudaEvent_t open_ev = nullptr;
    int open_phase = -1;

    // state flags
    bool have_particles = false, tree_valid = false, gravity_valid = false;
    bool sorted_valid = false;  // particles in Morton order for the current positions (keys, order)
    bool density_valid = false, force_valid = false, have_h = false, sphf_valid = false;
    bool use_pred = false;      // SPH uses predicted v, u (inside a KDK step)
    int last_grav_mode = -1;
    bool nbr_valid = false;   // neighbour lists of the current kernel-size search (not restored by gnb_load)
};

namespace gnb {

// host helpers (capi.cu)
int fail(gnb_ctx *c, int code, const std::string &msg);
int cuda_check(gnb_ctx *c, cudaError_t e, const char *what);
void dfree(gnb_ctx *c, void *p);

// Device allocation of count elements; GNB_ENOMEM on failure.
template <class T>
inline int dalloc(gnb_ctx *c, T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(c, GNB_ENOMEM, "device allocation of " + std::to_string(count * sizeof(T)) + " bytes failed");
    }
    return GNB_OK;
}

// phase timers (capi.cu): events recorded on the context stream around
// each phase, resolved after the call's final synchronisation
void phase_begin(gnb_ctx *c, int phase);
void phase_end(gnb_ctx *c);

// sort.cu
int morton_and_sort(gnb_ctx *c);
int radix_sort_pairs(gnb_ctx *c, uint64_t *k0, int *v0, uint64_t *k1, int *v1, int n, int first_digit);
// replace.cu
int replace_particles(gnb_ctx *c, int64_t n, const int64_t *id, const double *x, const double *y, const double *z,
                      const float *vx, const float *vy, const float *vz, const float *u, int on_device);
void replace_free(gnb_ctx *c);

// integrate.cu: hierarchical timesteps
int hier_buffers(gnb_ctx *c);
int hier_permute(gnb_ctx *c);
int hier_start(gnb_ctx *c, int K, double tick, double courant, double t_span);
int hier_predict(gnb_ctx *c, long long T, double tick);
int hier_update(gnb_ctx *c, long long T, int K, double tick, double courant, double t_span);
void hier_free(gnb_ctx *c);
int root_box(gnb_ctx *c);
// tree.cu
int build_tree(gnb_ctx *c, Tree &t, const uint64_t *skey, int n, const int *n_d, int n_leaf,
               int n_group, const int *pcx, const int *pcy, const int *pcz, const float *prx,
               const float *pry, const float *prz, const float *pm, const float *peps,
               bool moments);
int tree_alloc(gnb_ctx *c, Tree &t, int cap);
void tree_free(gnb_ctx *c, Tree &t);
int device_scan(gnb_ctx *c, const int *in, int *out, const int *n_d, int nmax, int *total_d);
int gas_slots(gnb_ctx *c, const uint8_t *type, const int *n_d, int *gslot);
int save_state(gnb_ctx *c, const char *path);
int load_state(gnb_ctx *c, const char *path);
// gravity.cu
int gravity_tree(gnb_ctx *c);
int gravity_direct(gnb_ctx *c);
int gravity_nfw(gnb_ctx *c);
// sph.cu
int sph_density(gnb_ctx *c);
int sph_force(gnb_ctx *c);
// surrogate.cu
int voxelise_buffers_for(gnb_ctx *c, int nreg, int grid);
int voxelise(gnb_ctx *c, int nreg, const double *centers, double side, int grid, float *out_dev);
int remap_regions(gnb_ctx *c, int nreg, const double *centers, double side, int grid, const float *pred_dev,
                  uint64_t seed, int sweeps);
// GNB_ETIMEOUT (and clears it) when a tensor-core convolution of the network
// recorded a bounded wait that ran out; the caller has synchronised.
int unet_poll_error(gnb_unet *u);
int sn_async_submit(gnb_ctx *c, gnb_unet *net, int nreg, const double *centers, double side, uint64_t seed,
                    int sweeps);
int sn_async_apply(gnb_ctx *c);
int sn_surrogate_batch(gnb_ctx *c, gnb_unet *net, int nreg, const double *centers, double side, uint64_t seed,
                       int sweeps, int use_graph);
// sn.cu
int inject_energy(gnb_ctx *c, const double pos[3], double E, double out[4]);
int cfl_min_h_over_vsig(gnb_ctx *c, double *out);
// integrate.cu
int kick(gnb_ctx *c, float hdt, bool gas_u);
int drift(gnb_ctx *c, double dt);
int predict(gnb_ctx *c, float hdt);
int kick_drift_predict(gnb_ctx *c, float hdt, double dt);
int diagnostics(gnb_ctx *c, double out[10]);
int scatter_out(gnb_ctx *c, int field, void *dst_dev);
int zero_forces(gnb_ctx *c);

}  // namespace gnb

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
#define GNB_LAUNCH_CHECK(c, what)                                                    \
    do {                                                                             \
        cudaError_t e_ = cudaGetLastError();                                         \
        if (e_ != cudaSuccess) return gnb::cuda_check((c), e_, (what));              \
    } while (0)

#define GNB_TRY(expr)                 \
    do {                              \
        int rc_ = (expr);             \
        if (rc_ != GNB_OK) return rc_; \
    } while (0)

__device__ __forceinline__ float fsqr(float a) { return a * a; }

// Offset of a particle from a reference grid point: the integer cell
// difference is exact in FP32 (|d| < 2^24) and scaling by the power-of-two
// unit is exact, so the FMA rounds once.
__device__ __forceinline__ float grid_off(int c, int cref, float r, float unit)
{
    return __fmaf_rn((float)(c - cref), unit, r);
}

template <class T>
__device__ __forceinline__ T warp_sum(T v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
