// Internal declarations shared by the libtreepm translation units.
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <cstdint>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "treepm.h"

namespace tpm {

constexpr int kMaxLevel = 21;  // 21 bits per axis, 63-bit keys
constexpr int kEwaldN = 64;    // Ewald correction table: kEwaldN intervals per axis over [0, L/2]

// ------------------------------------------------------------------ errors
void set_error(const char *fmt, ...);
void clear_error();

#define TPM_CUDA(call)                                                                                   \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) {                                                                         \
            ::tpm::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return TPM_ECUDA;                                                                            \
        }                                                                                                \
    } while (0)

#define TPM_CHECK(expr)            \
    do {                           \
        int s_ = (expr);           \
        if (s_ != TPM_OK)          \
            return s_;             \
    } while (0)

// ------------------------------------------------------------------ counters
// Kernels of this library launched since load (own kernels; CUB primitive
// invocations are counted separately, one per call).
void count_launch(int k = 1);
void count_cub_call(int k = 1);

// ------------------------------------------------------------------ memory
// Device memory drawn from the context's stream-ordered pool and counted
// against its HBM budget.
struct Ctx;

struct DevAlloc {
    void *p = nullptr;
    size_t bytes = 0;
};

int ctx_alloc(Ctx *c, void **p, size_t bytes, cudaStream_t st);
void ctx_free(Ctx *c, void *p, size_t bytes, cudaStream_t st);

// A set of allocations released together (a system, or one call's scratch).
struct AllocSet {
    Ctx *ctx = nullptr;
    std::vector<DevAlloc> list;
    template <class T>
    int get(T **p, size_t count, cudaStream_t st) {
        size_t b = count * sizeof(T);
        if (b == 0)
            b = 16;
        void *q = nullptr;
        int s = ctx_alloc(ctx, &q, b, st);
        if (s != TPM_OK)
            return s;
        list.push_back({q, b});
        *p = static_cast<T *>(q);
        return TPM_OK;
    }
    void release(cudaStream_t st) {
        for (auto &a : list)
            ctx_free(ctx, a.p, a.bytes, st);
        list.clear();
    }
    size_t bytes() const {
        size_t t = 0;
        for (auto &a : list)
            t += a.bytes;
        return t;
    }
};

// Several arrays carved from one allocation of an AllocSet (one pool call
// instead of one per array; each array starts on a 256-byte boundary).
struct Carve {
    struct Item {
        void *p;
        void (*set)(void *, char *);
        size_t off;
    };
    std::vector<Item> items;
    size_t total = 0;
    template <class T>
    static void set_ptr(void *pp, char *v) {
        *static_cast<T **>(pp) = reinterpret_cast<T *>(v);
    }
    template <class T>
    void add(T **p, size_t count) {
        size_t b = count * sizeof(T);
        if (b == 0)
            b = 16;
        items.push_back({static_cast<void *>(p), &set_ptr<T>, total});
        total += (b + 255) & ~size_t(255);
    }
    int commit(AllocSet &set, cudaStream_t st) {
        char *base = nullptr;
        const int rc = set.get(&base, total, st);
        if (rc != TPM_OK)
            return rc;
        for (auto &it : items)
            it.set(it.p, base + it.off);
        return TPM_OK;
    }
};

// ------------------------------------------------------------------ system
struct System {
    uint64_t id = 0;
    int64_t n = 0, nnodes = 0;
    tpm_build_params bp{};
    double x0[3] = {0, 0, 0}, L0 = 1.0;
    AllocSet mem;

    // particles
    double *pos = nullptr;   // n x 3 FP64 positions the tree uses (shifted / wrapped), original order
    float *mass = nullptr;   // n, original order
    uint64_t *key = nullptr; // n, sorted
    uint32_t *perm = nullptr;  // sorted position -> original index
    uint32_t *rank = nullptr;  // original index -> sorted position
    float4 *spart = nullptr;   // n, sorted: (x - leaf centre) FP32, mass
    // per-particle softening (Sec. 3.2), nullptr when uniform: spline support
    // per sorted particle, and per node its largest support, negative when
    // the node holds particles of different supports (pre-order and BFS)
    float *psoft = nullptr;
    float *nsoft = nullptr;
    float *bsoft = nullptr;

    // nodes, depth-first pre-order
    float4 *ncen = nullptr;  // geometric centre relative to x0 (exact in FP32), side L
    float4 *ncom = nullptr;  // centre of mass minus geometric centre (FP32), mass (FP32)
    int4 *nlink = nullptr;   // skip, first particle, count, leaf flag
    // the same nodes in breadth-first order (children of a node contiguous), for
    // the group walk: centre + side, centre of mass offset + mass, and
    // (first child, child count, first particle, particle count)
    float4 *bcen = nullptr;
    float4 *bcom = nullptr;
    int4 *blink = nullptr;
    uint8_t *nlevel = nullptr;
    uint64_t *nprefix = nullptr;
    // FP64 mass and mass-weighted position sums by breadth-first index, and
    // the pre-order -> breadth-first map (for export)
    double *msum = nullptr;
    double *ssum = nullptr;
    uint32_t *pre2bfs = nullptr;

    // device status word: bit 0 an active id was out of range, bit 1 the group
    // walk's candidate stack overflowed (read and cleared by tpm_sync_status)
    int *err = nullptr;

    double bb_lo[3] = {0, 0, 0}, bb_hi[3] = {0, 0, 0};  // bounding box of the tree positions

    // long-range mesh: potential and x, y, z force meshes of pm_mesh^3 points
    // (pm_mesh = pm_n, or 2 pm_n zero-padded for open boundaries) at
    // pm_corner + i pm_side / pm_n
    AllocSet pm_mem;
    float *phi = nullptr;
    // spectral gradient (periodic, TPM_GRAD_IK): x, y, z force meshes of
    // pm_mesh^3 points each, one after the other; null for the 4-point difference
    float *fmesh = nullptr;
    int pm_grad = TPM_GRAD_FD4;
    int pm_n = 0;
    int pm_mesh = 0;
    double pm_corner[3] = {0, 0, 0};
    double pm_rs = 0.0;
    double pm_G = 0.0;
};

constexpr size_t kPinnedStateBytes = 4096;

struct Ctx {
    int device = 0;
    void *pinned_state = nullptr;  // host page for a build's device-side bookkeeping
    std::mutex build_mu;
    // side stream of the tree build (work that overlaps the monopole pass) and
    // its fork / join events; used under build_mu
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_state = nullptr;  // a build's state has reached the pinned page
    int num_sms = 0;
    size_t budget = 0;
    size_t used = 0;
    cudaMemPool_t pool = nullptr;
    std::mutex mu;
    std::unordered_map<uint64_t, System *> systems;
    uint64_t next_id = 1;
    // cached cuFFT plans (one pair per mesh size)
    std::unordered_map<int, std::pair<cufftHandle, cufftHandle>> fft_plans;
    std::unordered_map<int, size_t> fft_work_bytes;
    // transforms of the isolated long-range kernel in mesh units, keyed by
    // (padded mesh size, split scale in cells)
    std::map<std::pair<int, double>, DevAlloc> iso_green;
    // Ewald correction of the periodic tree (unit box), and its value at d = 0
    DevAlloc ewald_tab;
    float ewald_phi0 = 0.0f;
};

// The context's Ewald correction table ((kEwaldN+1)^3 float4, unit box),
// built on first use unless may_alloc is false.
int ewald_table_for(Ctx *c, bool may_alloc, cudaStream_t st, const float4 **tab, float *phi0);

// Side of the mesh region: the box (periodic) or the tree root's side, a
// cube centred on the particles (open boundaries, zero-padded mesh).
inline double pm_side(const System *s) { return s->bp.periodic ? s->bp.box : s->L0; }

// ------------------------------------------------------------------ stages
// Tree build (keys, sort, levels, multipoles, pre-order tables): fills s.
int build_tree_device(Ctx *c, System *s, const double *pos_in, const float *mass_in, const float *hsoft_in,
                      cudaStream_t st);

// Long-range mesh potential into s->phi.
int pm_solve_device(Ctx *c, System *s, const tpm_force_params *p, cudaStream_t st);

struct WalkRequest {
    const uint32_t *sorted_idx;  // n_act sorted positions of the active particles, ascending
    const uint32_t *slot;        // n_act output slots
    const float *a_old;          // per slot (nullable)
    int64_t n_act;
    float *acc;                  // slot-major x 3
    float *pot;                  // nullable
    uint32_t *nint;              // nullable
    int accumulate;              // 1: add to acc / pot instead of overwriting
    int no_alloc = 0;            // 1: the call must not allocate device memory
    // open boundaries: room for n_act runs of spread-out chunks and their
    // count, for the lane walk (which hands them to the group walk; cleared by
    // walk_device)
    uint2 *runs = nullptr;
    unsigned *nruns = nullptr;
};

int walk_device(Ctx *c, const System *s, const tpm_force_params *p, const WalkRequest &r, cudaStream_t st);

// Batched walk (open boundaries): request descriptors are opaque records of
// batch_req_bytes() bytes filled by fill_batch_req; groups are (start, count,
// request, 0) over the sorted active list; group_size 64 takes the walk with
// two particles per lane (else groups of at most 32, one per lane);
// stack_depth is the candidate-stack capacity of the walk (128, 192 or 256).
size_t batch_req_bytes();
void fill_batch_req(void *dst, const System *s, const tpm_force_params *p);
int launch_walk_batch(Ctx *c, int group_size, int stack_depth, const void *reqs, const uint4 *groups,
                      const unsigned *n_groups, unsigned *next, const uint32_t *sidx, const uint32_t *slot,
                      const float *a_old, float *acc, float *pot, uint32_t *nint, int *err, cudaStream_t st);

// FP64 conservation diagnostics over all particles of s (device arrays in the
// caller's order): out_host[0..2] total force, [3] potential energy, [4]
// kinetic energy, [5..7] momentum, [8] sum of m |a|.  Synchronous.
constexpr int kDiagSums = 9;
int diagnostics_device(Ctx *c, const System *s, const float *acc, const float *pot, const double *vel,
                       double *out_host, cudaStream_t st);

// Adds the CIC-interpolated mesh force and potential to acc / pot.
int pm_interp_device(Ctx *c, const System *s, const WalkRequest &r, cudaStream_t st);

}  // namespace tpm
