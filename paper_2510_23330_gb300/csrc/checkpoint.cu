// checkpoint.cu -- save and restore of a context's particle state (the paper
// describes no checkpoint format; this is the library's own).
//
// File: a 128-byte header, then arrays of n entries in the caller's particle
// order (the order of the last gnb_set_particles), little-endian as the
// host writes them:
//   header  "GNBSTAT1", uint32 version (1), uint32 flags, int64 n, int64 n_gas,
//           int32 last gravity mode, zero padding to 128 bytes;
//   state   id int64, type uint8, x y z float64, vx vy vz m eps u float32,
//           h2 float64 (0 for stars and before the first kernel-size search);
//   results ax ay az pot pot_ext agrav_x agrav_y agrav_z dudt rho pres cs
//           float32 (those of the last force evaluation; which of them are
//           current is in the flags).
// Loading goes through the same path as gnb_set_particles (validation, the
// caller order as slot order) and then restores the supports and results
// with their validity flags, so a KDK integration resumed from the file
// kicks with the same accelerations and sorts into the same order as the
// context that wrote it.
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace gnb {

namespace {

constexpr char CK_MAGIC[8] = {'G', 'N', 'B', 'S', 'T', 'A', 'T', '1'};
constexpr unsigned CK_VERSION = 1;
enum : unsigned {
    CK_HAVE_H = 1,
    CK_FORCE = 2,
    CK_GRAVITY = 4,
    CK_DENSITY = 8,
    CK_SPHF = 16,
};

struct CkHeader {
    char magic[8];
    uint32_t version, flags;
    int64_t n, n_gas;
    int32_t grav_mode;
    unsigned char pad[128 - 8 - 8 - 16 - 4];
};
static_assert(sizeof(CkHeader) == 128, "checkpoint header is 128 bytes");

template <class T>
__global__ void k_ck_out(const T *__restrict__ src, const int *__restrict__ orig, int n, T *__restrict__ dst)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[orig[i]] = src[i];
}

struct File {
    FILE *f = nullptr;
    ~File() { if (f) fclose(f); }
};

// one per-slot array to caller order, through the export staging buffer, to the file
template <class T>
int write_array(gnb_ctx *c, FILE *f, const T *src, std::vector<unsigned char> &host)
{
    const int n = (int)c->n;
    T *stage = reinterpret_cast<T *>(c->tmp_out);
    counted(k_ck_out<T>)<<<(n + 255) / 256, 256, 0, c->s>>>(src, c->P[c->cur].orig, n, stage);
    GNB_LAUNCH_CHECK(c, "checkpoint gather");
    const size_t bytes = sizeof(T) * (size_t)n;
    host.resize(bytes);
    GNB_TRY(cuda_check(c, cudaMemcpyAsync(host.data(), stage, bytes, cudaMemcpyDeviceToHost, c->s), "checkpoint copy"));
    GNB_TRY(cuda_check(c, cudaStreamSynchronize(c->s), "checkpoint sync"));
    if (fwrite(host.data(), 1, bytes, f) != bytes) return fail(c, GNB_EINVAL, "checkpoint write failed");
    return GNB_OK;
}

template <class T>
bool read_array(FILE *f, std::vector<T> &v, int64_t n)
{
    v.resize((size_t)n);
    return fread(v.data(), sizeof(T), (size_t)n, f) == (size_t)n;
}

template <class T>
int to_device(gnb_ctx *c, T *dst, const std::vector<T> &v)
{
    return cuda_check(c, cudaMemcpyAsync(dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, c->s),
                      "checkpoint restore");
}

}  // namespace

int save_state(gnb_ctx *c, const char *path)
{
    File F;
    F.f = fopen(path, "wb");
    if (!F.f) return fail(c, GNB_EINVAL, std::string("cannot open for writing: ") + path);
    CkHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, CK_MAGIC, 8);
    h.version = CK_VERSION;
    h.flags = (c->have_h ? CK_HAVE_H : 0) | (c->force_valid ? CK_FORCE : 0) | (c->gravity_valid ? CK_GRAVITY : 0) |
              (c->density_valid ? CK_DENSITY : 0) | (c->sphf_valid ? CK_SPHF : 0);
    h.n = c->n;
    h.n_gas = c->n_gas;
    h.grav_mode = c->last_grav_mode;
    if (fwrite(&h, sizeof(h), 1, F.f) != 1) return fail(c, GNB_EINVAL, "checkpoint write failed");
    std::vector<unsigned char> host;
    const PArr &p = c->P[c->cur];
    GNB_TRY(write_array(c, F.f, p.id, host));
    GNB_TRY(write_array(c, F.f, p.type, host));
    for (const double *a : {p.x, p.y, p.z}) GNB_TRY(write_array(c, F.f, a, host));
    for (const float *a : {p.vx, p.vy, p.vz, p.m, p.eps, p.u}) GNB_TRY(write_array(c, F.f, a, host));
    GNB_TRY(write_array(c, F.f, p.h2, host));
    for (const float *a : {c->ax, c->ay, c->az, c->pot, c->pext, c->gax, c->gay, c->gaz, c->dudt, c->rho, c->pres,
                           c->cs})
        GNB_TRY(write_array(c, F.f, a, host));
    if (fflush(F.f) != 0) return fail(c, GNB_EINVAL, "checkpoint write failed");
    return GNB_OK;
}

int load_state(gnb_ctx *c, const char *path)
{
    File F;
    F.f = fopen(path, "rb");
    if (!F.f) return fail(c, GNB_EINVAL, std::string("cannot open for reading: ") + path);
    CkHeader h;
    if (fread(&h, sizeof(h), 1, F.f) != 1 || memcmp(h.magic, CK_MAGIC, 8) != 0)
        return fail(c, GNB_EINVAL, "not a galnb state file");
    if (h.version != CK_VERSION) return fail(c, GNB_EINVAL, "unsupported state file version");
    if (h.n < 1 || h.n > (1ll << 30)) return fail(c, GNB_EINVAL, "state file particle count out of range");
    const int64_t n = h.n;
    std::vector<int64_t> id;
    std::vector<uint8_t> type;
    std::vector<double> x, y, z, h2;
    std::vector<float> vx, vy, vz, m, eps, u;
    std::vector<float> res[12];
    bool ok = read_array(F.f, id, n) && read_array(F.f, type, n) && read_array(F.f, x, n) && read_array(F.f, y, n) &&
              read_array(F.f, z, n) && read_array(F.f, vx, n) && read_array(F.f, vy, n) && read_array(F.f, vz, n) &&
              read_array(F.f, m, n) && read_array(F.f, eps, n) && read_array(F.f, u, n) && read_array(F.f, h2, n);
    for (auto &r : res) ok = ok && read_array(F.f, r, n);
    if (!ok) return fail(c, GNB_EINVAL, "state file truncated");
    const int rc = gnb_set_particles(c, n, id.data(), type.data(), x.data(), y.data(), z.data(), vx.data(), vy.data(),
                                     vz.data(), m.data(), eps.data(), u.data(), 0);
    if (rc != GNB_OK) return rc;
    if (c->n_gas != h.n_gas) return fail(c, GNB_EMISMATCH, "state file gas count differs from its particles");
    // after gnb_set_particles the slots are in caller order
    GNB_TRY(to_device(c, c->P[c->cur].h2, h2));
    float *dst[12] = {c->ax, c->ay, c->az, c->pot, c->pext, c->gax, c->gay, c->gaz, c->dudt, c->rho, c->pres, c->cs};
    for (int k = 0; k < 12; k++) GNB_TRY(to_device(c, dst[k], res[k]));
    GNB_TRY(cuda_check(c, cudaStreamSynchronize(c->s), "checkpoint restore sync"));
    c->have_h = (h.flags & CK_HAVE_H) != 0;
    c->force_valid = (h.flags & CK_FORCE) != 0;
    c->gravity_valid = (h.flags & CK_GRAVITY) != 0;
    c->density_valid = (h.flags & CK_DENSITY) != 0;
    c->sphf_valid = (h.flags & CK_SPHF) != 0;
    c->nbr_valid = false;  // the neighbour lists are not in the file
    c->last_grav_mode = h.grav_mode;
    return GNB_OK;
}

}  // namespace gnb
