// libtreepm runtime: contexts, the HBM-budgeted device memory pool, the
// registry of resident systems, host/device argument marshalling and the
// extern "C" entry points declared in treepm.h.
#include <cub/cub.cuh>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstring>

#include "tpm_internal.cuh"

namespace tpm {

// ------------------------------------------------------------------ errors
namespace {
thread_local char g_err[512] = "";
}

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}
void clear_error() { g_err[0] = 0; }

namespace {
std::atomic<unsigned long long> g_launches{0}, g_cub_calls{0};
}
void count_launch(int k) { g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed); }
void count_cub_call(int k) { g_cub_calls.fetch_add((unsigned long long)k, std::memory_order_relaxed); }

// ------------------------------------------------------------------ memory
namespace {
std::mutex g_acct_mu;
}

int ctx_alloc(Ctx *c, void **p, size_t bytes, cudaStream_t st) {
    bytes = (bytes + 255) & ~size_t(255);
    {
        std::lock_guard<std::mutex> lk(g_acct_mu);
        if (c->used + bytes > c->budget) {
            set_error("HBM budget exceeded: %zu bytes in use + %zu requested > budget %zu", c->used, bytes,
                      c->budget);
            return TPM_EBUDGET;
        }
        c->used += bytes;
    }
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, c->pool, st);
    if (e != cudaSuccess) {
        std::lock_guard<std::mutex> lk(g_acct_mu);
        c->used -= bytes;
        set_error("cudaMallocFromPoolAsync(%zu) failed: %s", bytes, cudaGetErrorString(e));
        return TPM_ECUDA;
    }
    return TPM_OK;
}

void ctx_free(Ctx *c, void *p, size_t bytes, cudaStream_t st) {
    if (!p)
        return;
    bytes = (bytes + 255) & ~size_t(255);
    cudaFreeAsync(p, st);
    std::lock_guard<std::mutex> lk(g_acct_mu);
    c->used -= std::min(bytes, c->used);
}

namespace {

// Host argument checks: a branch-free pass over fixed-size blocks (which the
// compiler vectorises), and a scan of the one block that fails for the index
// reported.  The index of the first failing element, or -1.
constexpr int64_t kCheckBlock = 4096;

template <class Bad, class T>
int64_t first_failing(const T *x, int64_t n, Bad bad) {
    int64_t b = 0;
    for (; b + kCheckBlock <= n; b += kCheckBlock) {
        const T *blk = x + b;
        unsigned any = 0u;
        for (int64_t k = 0; k < kCheckBlock; k++)
            any |= bad(blk[k]) ? 1u : 0u;
        if (any)
            break;
    }
    for (int64_t k = b; k < n; k++)
        if (bad(x[k]))
            return k;
    return -1;
}

// non-finite: all exponent bits set (infinity or NaN)
inline bool nonfinite_bits(float v) {
    uint32_t u;
    memcpy(&u, &v, sizeof u);
    return (u & 0x7f800000u) == 0x7f800000u;
}

bool is_device_ptr(const void *p) {
    if (!p)
        return false;
    cudaPointerAttributes a{};
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Address through which kernels reach p: device or managed memory as it is;
// page-locked host memory through its mapped device address (kernels read it
// in place across the coherent CPU-GPU link, no staging copy); nullptr for
// pageable host memory.  Used for the tree build's inputs, each read once in
// a coalesced stream; the force call stages its host arguments (per-group
// reads of a_old and scattered writes of results in place cost more than one
// bulk copy each way).
const void *device_view(const void *p) {
    if (!p)
        return nullptr;
    cudaPointerAttributes a{};
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)
        return p;
    if (a.type == cudaMemoryTypeHost && a.devicePointer)
        return a.devicePointer;
    return nullptr;
}

System *find(Ctx *c, tpm_sys id) {
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->systems.find(id);
    return it == c->systems.end() ? nullptr : it->second;
}

int check_force_params(const System *s, const tpm_force_params *p) {
    if (!p) {
        set_error("null force params");
        return TPM_EINVAL;
    }
    if (p->crit != TPM_CRIT_BH && p->crit != TPM_CRIT_RELATIVE) {
        set_error("crit must be TPM_CRIT_BH or TPM_CRIT_RELATIVE");
        return TPM_EINVAL;
    }
    if (p->crit == TPM_CRIT_BH && !(p->theta > 0.0 && std::isfinite(p->theta))) {
        set_error("theta must be finite and > 0");
        return TPM_EINVAL;
    }
    if (p->crit == TPM_CRIT_RELATIVE && !(p->alpha >= 0.0 && std::isfinite(p->alpha))) {
        set_error("alpha must be finite and >= 0");
        return TPM_EINVAL;
    }
    if (p->plain_fp32 != 0 && p->plain_fp32 != 1) {
        set_error("plain_fp32 must be 0 or 1");
        return TPM_EINVAL;
    }
    if (p->plain_fp32 && s && s->bp.periodic) {
        set_error("the plain FP32 form is available for open boundaries");
        return TPM_EINVAL;
    }
    if (p->treepm) {
        int n = p->pm_n;
        const int nmax = (s && !s->bp.periodic) ? 512 : 1024;  // open boundaries: a (2 n)^3 padded mesh
        if (n < 8 || n > nmax || (n & (n - 1))) {
            set_error("pm_n must be a power of two in [8, %d]", nmax);
            return TPM_EINVAL;
        }
        if (!(p->asmth > 0.0) || !(p->rcut > 0.0) || !std::isfinite(p->asmth) || !std::isfinite(p->rcut)) {
            set_error("asmth and rcut must be finite and > 0");
            return TPM_EINVAL;
        }
        if (s && s->bp.periodic && p->rcut * p->asmth * s->bp.box / n >= 0.25 * s->bp.box) {
            set_error("cutoff radius must stay below a quarter of the box");
            return TPM_EINVAL;
        }
        if (p->pm_grad != TPM_GRAD_FD4 && p->pm_grad != TPM_GRAD_IK) {
            set_error("pm_grad must be TPM_GRAD_FD4 or TPM_GRAD_IK");
            return TPM_EINVAL;
        }
        if (s && !s->bp.periodic && p->pm_grad != TPM_GRAD_FD4) {
            set_error("the spectral mesh gradient is available for periodic systems");
            return TPM_EINVAL;
        }
    }
    return TPM_OK;
}

// Sort keys of the active set: each id's sorted position in the tree, with its
// slot in the caller's order.  An id out of range sets bit 0 of the system's
// status word and is read as particle 0, so every access stays in bounds.
__global__ void k_active_keys(const uint32_t *__restrict__ ids, int64_t n_act, const uint32_t *__restrict__ rank,
                              int64_t n, uint32_t *__restrict__ keys, uint32_t *__restrict__ vals,
                              int *__restrict__ bad) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n_act)
        return;
    uint32_t id = ids[k];
    if (id >= (uint64_t)n) {
        atomicOr(bad, 1);
        id = 0;
    }
    keys[k] = rank[id];
    vals[k] = (uint32_t)k;
}

int key_bits(int64_t n) {
    int b = 1;
    while ((int64_t(1) << b) < n)
        b++;
    return b;
}

}  // namespace
}  // namespace tpm

using namespace tpm;

extern "C" {

int tpm_version(void) { return TPM_API_VERSION; }

const char *tpm_last_error(void) { return g_err; }

int tpm_launch_counts(uint64_t *kernels, uint64_t *cub_calls) {
    if (kernels)
        *kernels = g_launches.load();
    if (cub_calls)
        *cub_calls = g_cub_calls.load();
    return TPM_OK;
}

int tpm_create(tpm_ctx **out, int device, size_t budget) {
    clear_error();
    if (!out) {
        set_error("null ctx pointer");
        return TPM_EINVAL;
    }
    *out = nullptr;
    int ndev = 0;
    TPM_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) {
        set_error("device %d out of range (%d devices)", device, ndev);
        return TPM_EINVAL;
    }
    TPM_CUDA(cudaSetDevice(device));
    Ctx *c = new Ctx;
    c->device = device;
    cudaDeviceProp prop{};
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) {
        delete c;
        set_error("cudaGetDeviceProperties: %s", cudaGetErrorString(e));
        return TPM_ECUDA;
    }
    c->num_sms = prop.multiProcessorCount;
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    c->budget = budget ? budget : (size_t)(0.9 * (double)fr);
    cudaMemPoolProps pp{};
    pp.allocType = cudaMemAllocationTypePinned;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = device;
    e = cudaMemPoolCreate(&c->pool, &pp);
    if (e != cudaSuccess) {
        delete c;
        set_error("cudaMemPoolCreate: %s", cudaGetErrorString(e));
        return TPM_ECUDA;
    }
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    e = cudaMallocHost(&c->pinned_state, kPinnedStateBytes);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&c->ev_state, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        if (c->ev_fork)
            cudaEventDestroy(c->ev_fork);
        if (c->ev_join)
            cudaEventDestroy(c->ev_join);
        if (c->side)
            cudaStreamDestroy(c->side);
        if (c->pinned_state)
            cudaFreeHost(c->pinned_state);
        cudaMemPoolDestroy(c->pool);
        delete c;
        set_error("context setup: %s", cudaGetErrorString(e));
        return TPM_ECUDA;
    }
    *out = reinterpret_cast<tpm_ctx *>(c);
    return TPM_OK;
}

int tpm_destroy(tpm_ctx *h) {
    clear_error();
    if (!h)
        return TPM_OK;
    Ctx *c = reinterpret_cast<Ctx *>(h);
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (auto &kv : c->systems) {
        kv.second->pm_mem.release(0);
        kv.second->mem.release(0);
        delete kv.second;
    }
    c->systems.clear();
    for (auto &kv : c->fft_plans) {
        cufftDestroy(kv.second.first);
        cufftDestroy(kv.second.second);
    }
    for (auto &kv : c->iso_green)
        ctx_free(c, kv.second.p, kv.second.bytes, 0);
    c->iso_green.clear();
    ctx_free(c, c->ewald_tab.p, c->ewald_tab.bytes, 0);
    cudaStreamSynchronize(0);
    cudaMemPoolDestroy(c->pool);
    cudaFreeHost(c->pinned_state);
    cudaEventDestroy(c->ev_fork);
    cudaEventDestroy(c->ev_join);
    cudaEventDestroy(c->ev_state);
    cudaStreamDestroy(c->side);
    delete c;
    return TPM_OK;
}

int tpm_memory(const tpm_ctx *h, size_t *used, size_t *budget) {
    clear_error();
    if (!h) {
        set_error("null ctx");
        return TPM_EINVAL;
    }
    const Ctx *c = reinterpret_cast<const Ctx *>(h);
    std::lock_guard<std::mutex> lk(g_acct_mu);
    if (used)
        *used = c->used;
    if (budget)
        *budget = c->budget;
    return TPM_OK;
}

}  // extern "C"

namespace tpm {
namespace {

int build_entry(tpm_ctx *h, const double *pos, const float *mass, const float *hsoft, int64_t n,
                const tpm_build_params *p, void *stream, tpm_sys *out) {
    if (!h || !pos || !mass || !p || !out) {
        set_error("null argument");
        return TPM_EINVAL;
    }
    if (n < 1 || n > 0x7fffffffLL) {
        set_error("n must lie in [1, 2^31 - 1]");
        return TPM_EINVAL;
    }
    if (!(p->G > 0.0) || !(p->h > 0.0) || p->leaf_bucket < 1 || !std::isfinite(p->G) || !std::isfinite(p->h)) {
        set_error("G and h must be finite and > 0, leaf_bucket >= 1");
        return TPM_EINVAL;
    }
    if (p->periodic && !(p->box > 0.0 && std::isfinite(p->box))) {
        set_error("periodic box must be finite and > 0");
        return TPM_EINVAL;
    }
    for (int a = 0; a < 3; a++)
        if (!(p->shift[a] >= 0.0 && p->shift[a] < 1.0)) {
            set_error("shift must lie in [0, 1)");
            return TPM_EINVAL;
        }
    Ctx *c = reinterpret_cast<Ctx *>(h);
    TPM_CUDA(cudaSetDevice(c->device));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    System *s = new System;
    s->mem.ctx = c;
    s->pm_mem.ctx = c;
    s->n = n;
    s->bp = *p;
    AllocSet stage;
    stage.ctx = c;
    const double *dpos = static_cast<const double *>(device_view(pos));
    const float *dmass = static_cast<const float *>(device_view(mass));
    int rc = TPM_OK;
    if (!dpos) {
        double *d = nullptr;
        rc = stage.get(&d, 3 * n, st);
        if (rc == TPM_OK && cudaMemcpyAsync(d, pos, 3 * n * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess) {
            set_error("copy of positions to the device failed");
            rc = TPM_ECUDA;
        }
        dpos = d;
    }
    if (rc == TPM_OK && !dmass) {
        float *d = nullptr;
        rc = stage.get(&d, n, st);
        if (rc == TPM_OK && cudaMemcpyAsync(d, mass, n * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess) {
            set_error("copy of masses to the device failed");
            rc = TPM_ECUDA;
        }
        dmass = d;
    }
    const float *dsoft = static_cast<const float *>(device_view(hsoft));
    if (rc == TPM_OK && hsoft && !dsoft) {
        float *d = nullptr;
        rc = stage.get(&d, n, st);
        if (rc == TPM_OK && cudaMemcpyAsync(d, hsoft, n * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess) {
            set_error("copy of softening lengths to the device failed");
            rc = TPM_ECUDA;
        }
        dsoft = d;
    }
    if (rc == TPM_OK)
        rc = build_tree_device(c, s, dpos, dmass, dsoft, st);
    stage.release(st);
    if (rc != TPM_OK) {
        s->mem.release(st);
        delete s;
        return rc;
    }
    std::lock_guard<std::mutex> lk(c->mu);
    s->id = c->next_id++;
    c->systems[s->id] = s;
    *out = s->id;
    return TPM_OK;
}

}  // namespace
}  // namespace tpm

extern "C" {

int tpm_build_tree(tpm_ctx *h, const double *pos, const float *mass, int64_t n, const tpm_build_params *p,
                   void *stream, tpm_sys *out) {
    clear_error();
    return build_entry(h, pos, mass, nullptr, n, p, stream, out);
}

int tpm_build_tree_soft(tpm_ctx *h, const double *pos, const float *mass, const float *hsoft, int64_t n,
                        const tpm_build_params *p, void *stream, tpm_sys *out) {
    clear_error();
    if (!hsoft) {
        set_error("null hsoft");
        return TPM_EINVAL;
    }
    if (p && p->periodic) {
        set_error("per-particle softening is available with open boundaries");
        return TPM_EINVAL;
    }
    return build_entry(h, pos, mass, hsoft, n, p, stream, out);
}

int tpm_pm_long_range(tpm_ctx *h, tpm_sys sid, const tpm_force_params *p, void *stream) {
    clear_error();
    if (!h) {
        set_error("null ctx");
        return TPM_EINVAL;
    }
    Ctx *c = reinterpret_cast<Ctx *>(h);
    System *s = find(c, sid);
    if (!s) {
        set_error("unknown system handle %llu", (unsigned long long)sid);
        return TPM_ENOSYS_HANDLE;
    }
    TPM_CHECK(check_force_params(s, p));
    if (!p->treepm) {
        set_error("tpm_pm_long_range needs treepm = 1");
        return TPM_EINVAL;
    }
    TPM_CUDA(cudaSetDevice(c->device));
    return pm_solve_device(c, s, p, reinterpret_cast<cudaStream_t>(stream));
}

int tpm_compute_forces(tpm_ctx *h, tpm_sys sid, const uint32_t *active_ids, int64_t n_active, const float *a_old,
                       const tpm_force_params *p, float *acc, float *pot, uint32_t *n_int, void *stream) {
    clear_error();
    if (!h || (!acc && n_active != 0)) {
        set_error("null argument");
        return TPM_EINVAL;
    }
    Ctx *c = reinterpret_cast<Ctx *>(h);
    System *s = find(c, sid);
    if (!s) {
        set_error("unknown system handle %llu", (unsigned long long)sid);
        return TPM_ENOSYS_HANDLE;
    }
    TPM_CHECK(check_force_params(s, p));
    if (n_active < 0 || n_active > s->n) {
        set_error("n_active must lie in [0, n]");
        return TPM_EINVAL;
    }
    if (n_active == 0)  // an empty active set: nothing to compute (its arrays may be null)
        return TPM_OK;
    if (!active_ids && n_active != s->n) {
        set_error("active_ids = NULL means all particles: n_active must equal n");
        return TPM_EINVAL;
    }
    if (p->crit == TPM_CRIT_RELATIVE && !a_old) {
        set_error("the relative criterion needs a_old");
        return TPM_EINVAL;
    }
    if (p->treepm) {
        const double rs = p->asmth * pm_side(s) / p->pm_n;
        if (!s->phi || s->pm_n != p->pm_n || std::fabs(s->pm_rs - rs) > 1e-12 * rs || s->pm_G != s->bp.G ||
            s->pm_grad != p->pm_grad) {
            set_error("no long-range mesh for these parameters: call tpm_pm_long_range first");
            return TPM_EINVAL;
        }
    }
    TPM_CUDA(cudaSetDevice(c->device));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

    const bool ids_dev = is_device_ptr(active_ids), aold_dev = is_device_ptr(a_old);
    const bool acc_dev = is_device_ptr(acc), pot_dev = is_device_ptr(pot), nint_dev = is_device_ptr(n_int);
    if (active_ids && !ids_dev) {
        const uint32_t lim = (uint32_t)s->n;  // n < 2^31 (checked when the tree was built)
        const int64_t k = first_failing(active_ids, n_active, [lim](uint32_t v) { return v >= lim; });
        if (k >= 0) {
            set_error("active_ids[%lld] = %u out of range", (long long)k, active_ids[k]);
            return TPM_EINVAL;
        }
    }
    if (a_old && !aold_dev && p->crit == TPM_CRIT_RELATIVE) {
        const int64_t k = first_failing(a_old, n_active, nonfinite_bits);
        if (k >= 0) {
            set_error("a_old[%lld] is not finite", (long long)k);
            return TPM_ENAN;
        }
    }

    AllocSet tmp;
    tmp.ctx = c;
    struct Guard {
        AllocSet &t;
        cudaStream_t st;
        ~Guard() { t.release(st); }
    } guard{tmp, st};

    // inputs on the device
    const uint32_t *d_ids = active_ids;
    const float *d_aold = (p->crit == TPM_CRIT_RELATIVE) ? a_old : nullptr;
    if (active_ids && !ids_dev) {
        uint32_t *d;
        TPM_CHECK(tmp.get(&d, n_active, st));
        TPM_CUDA(cudaMemcpyAsync(d, active_ids, n_active * 4, cudaMemcpyHostToDevice, st));
        d_ids = d;
    }
    if (d_aold && !aold_dev) {
        float *d;
        TPM_CHECK(tmp.get(&d, n_active, st));
        TPM_CUDA(cudaMemcpyAsync(d, a_old, n_active * 4, cudaMemcpyHostToDevice, st));
        d_aold = d;
    }
    // outputs on the device
    float *d_acc = acc, *d_pot = pot;
    uint32_t *d_nint = n_int;
    if (!acc_dev)
        TPM_CHECK(tmp.get(&d_acc, 3 * n_active, st));
    if (pot && !pot_dev)
        TPM_CHECK(tmp.get(&d_pot, n_active, st));
    if (n_int && !nint_dev)
        TPM_CHECK(tmp.get(&d_nint, n_active, st));

    // active set in key order
    WalkRequest r{};
    r.n_act = n_active;
    r.a_old = d_aold;
    r.acc = d_acc;
    r.pot = d_pot;
    r.nint = d_nint;
    if (d_ids) {
        uint32_t *keys, *vals, *sk, *sv;
        TPM_CHECK(tmp.get(&keys, n_active, st));
        TPM_CHECK(tmp.get(&vals, n_active, st));
        TPM_CHECK(tmp.get(&sk, n_active, st));
        TPM_CHECK(tmp.get(&sv, n_active, st));
        k_active_keys<<<(unsigned)((n_active + 255) / 256), 256, 0, st>>>(d_ids, n_active, s->rank, s->n, keys, vals,
                                                                         s->err);
        count_launch();
        TPM_CUDA(cudaGetLastError());
        size_t sb = 0;
        int bits = key_bits(s->n);
        TPM_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, sb, keys, sk, vals, sv, (int)n_active, 0, bits, st));
        void *cub_tmp;
        TPM_CHECK(tmp.get((char **)&cub_tmp, sb, st));
        TPM_CUDA(cub::DeviceRadixSort::SortPairs(cub_tmp, sb, keys, sk, vals, sv, (int)n_active, 0, bits, st));
        count_cub_call();
        r.sorted_idx = sk;
        r.slot = sv;
    }
    if (!s->bp.periodic) {  // runs of spread-out chunks
        TPM_CHECK(tmp.get(&r.runs, n_active, st));
        TPM_CHECK(tmp.get(&r.nruns, 1, st));
    }
    if (p->treepm) {
        TPM_CHECK(pm_interp_device(c, s, r, st));
        r.accumulate = 1;
    }
    TPM_CHECK(walk_device(c, s, p, r, st));

    bool sync = false;
    if (!acc_dev) {
        TPM_CUDA(cudaMemcpyAsync(acc, d_acc, 3 * n_active * sizeof(float), cudaMemcpyDeviceToHost, st));
        sync = true;
    }
    if (pot && !pot_dev) {
        TPM_CUDA(cudaMemcpyAsync(pot, d_pot, n_active * sizeof(float), cudaMemcpyDeviceToHost, st));
        sync = true;
    }
    if (n_int && !nint_dev) {
        TPM_CUDA(cudaMemcpyAsync(n_int, d_nint, n_active * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        sync = true;
    }
    // host inputs were staged asynchronously: keep them alive until copied
    const bool staged = (active_ids && !ids_dev) || (d_aold && !aold_dev);
    if (sync || staged)
        TPM_CUDA(cudaStreamSynchronize(st));
    return TPM_OK;
}

int tpm_diagnostics(tpm_ctx *h, tpm_sys sid, const float *acc, const float *pot, const double *vel, double *out,
                    void *stream) {
    clear_error();
    if (!h || !acc || !out) {
        set_error("null ctx, acc or out");
        return TPM_EINVAL;
    }
    Ctx *c = reinterpret_cast<Ctx *>(h);
    System *s = find(c, sid);
    if (!s) {
        set_error("unknown system handle %llu", (unsigned long long)sid);
        return TPM_ENOSYS_HANDLE;
    }
    if (!is_device_ptr(acc) || (pot && !is_device_ptr(pot)) || (vel && !is_device_ptr(vel))) {
        set_error("acc, pot and vel must be device arrays");
        return TPM_EINVAL;
    }
    TPM_CUDA(cudaSetDevice(c->device));
    return diagnostics_device(c, s, acc, pot, vel, out, reinterpret_cast<cudaStream_t>(stream));
}

int tpm_sync_status(tpm_ctx *h, tpm_sys sid, void *stream) {
    clear_error();
    if (!h) {
        set_error("null ctx");
        return TPM_EINVAL;
    }
    Ctx *c = reinterpret_cast<Ctx *>(h);
    System *s = find(c, sid);
    if (!s) {
        set_error("unknown system handle %llu", (unsigned long long)sid);
        return TPM_ENOSYS_HANDLE;
    }
    TPM_CUDA(cudaSetDevice(c->device));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int word = 0;
    TPM_CUDA(cudaMemcpyAsync(&word, s->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    TPM_CUDA(cudaStreamSynchronize(st));
    if (word == 0)
        return TPM_OK;
    TPM_CUDA(cudaMemsetAsync(s->err, 0, sizeof(int), st));
    TPM_CUDA(cudaStreamSynchronize(st));
    if (word & 1) {
        set_error("an active id was out of range (its outputs are those of particle 0)");
        return TPM_EINVAL;
    }
    set_error("the walk's candidate stack overflowed (device status %d)", word);
    return TPM_ECUDA;
}

int tpm_release(tpm_ctx *h, tpm_sys sid) {
    clear_error();
    if (!h) {
        set_error("null ctx");
        return TPM_EINVAL;
    }
    Ctx *c = reinterpret_cast<Ctx *>(h);
    System *s = nullptr;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        auto it = c->systems.find(sid);
        if (it == c->systems.end()) {
            set_error("unknown system handle %llu", (unsigned long long)sid);
            return TPM_ENOSYS_HANDLE;
        }
        s = it->second;
        c->systems.erase(it);
    }
    TPM_CUDA(cudaSetDevice(c->device));
    TPM_CUDA(cudaDeviceSynchronize());
    s->pm_mem.release(0);
    s->mem.release(0);
    delete s;
    return TPM_OK;
}

int tpm_tree_info(tpm_ctx *h, tpm_sys sid, int64_t *n, int64_t *nn, double *x0, double *L0) {
    clear_error();
    if (!h) {
        set_error("null ctx");
        return TPM_EINVAL;
    }
    System *s = find(reinterpret_cast<Ctx *>(h), sid);
    if (!s) {
        set_error("unknown system handle %llu", (unsigned long long)sid);
        return TPM_ENOSYS_HANDLE;
    }
    if (n)
        *n = s->n;
    if (nn)
        *nn = s->nnodes;
    if (x0)
        for (int a = 0; a < 3; a++)
            x0[a] = s->x0[a];
    if (L0)
        *L0 = s->L0;
    return TPM_OK;
}

int tpm_tree_export(tpm_ctx *h, tpm_sys sid, uint64_t *key, uint32_t *perm, uint8_t *level, uint64_t *prefix,
                    uint32_t *first, uint32_t *count, uint32_t *skip, double *mass, double *com, double *xtree) {
    clear_error();
    if (!h) {
        set_error("null ctx");
        return TPM_EINVAL;
    }
    Ctx *c = reinterpret_cast<Ctx *>(h);
    System *s = find(c, sid);
    if (!s) {
        set_error("unknown system handle %llu", (unsigned long long)sid);
        return TPM_ENOSYS_HANDLE;
    }
    TPM_CUDA(cudaSetDevice(c->device));
    TPM_CUDA(cudaDeviceSynchronize());
    const int64_t n = s->n, m = s->nnodes;
    if (key)
        TPM_CUDA(cudaMemcpy(key, s->key, n * 8, cudaMemcpyDeviceToHost));
    if (perm)
        TPM_CUDA(cudaMemcpy(perm, s->perm, n * 4, cudaMemcpyDeviceToHost));
    if (level)
        TPM_CUDA(cudaMemcpy(level, s->nlevel, m, cudaMemcpyDeviceToHost));
    if (prefix)
        TPM_CUDA(cudaMemcpy(prefix, s->nprefix, m * 8, cudaMemcpyDeviceToHost));
    if (mass || com) {
        // FP64 sums by breadth-first index; the centre of mass is S / m
        // (IEEE division, correctly rounded as on the device)
        std::vector<double> M(m), S(3 * m);
        std::vector<uint32_t> q(m);
        TPM_CUDA(cudaMemcpy(M.data(), s->msum, m * 8, cudaMemcpyDeviceToHost));
        TPM_CUDA(cudaMemcpy(S.data(), s->ssum, 3 * m * 8, cudaMemcpyDeviceToHost));
        TPM_CUDA(cudaMemcpy(q.data(), s->pre2bfs, m * 4, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < m; i++) {
            const double mi = M[q[i]];
            if (mass)
                mass[i] = mi;
            if (com)
                for (int a = 0; a < 3; a++)
                    com[3 * i + a] = S[3 * (size_t)q[i] + a] / mi;
        }
    }
    if (xtree)
        TPM_CUDA(cudaMemcpy(xtree, s->pos, 3 * n * 8, cudaMemcpyDeviceToHost));
    if (first || count || skip) {
        std::vector<int4> l(m);
        TPM_CUDA(cudaMemcpy(l.data(), s->nlink, m * sizeof(int4), cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < m; i++) {
            if (skip)
                skip[i] = (uint32_t)l[i].x;
            if (first)
                first[i] = (uint32_t)l[i].y;
            if (count)
                count[i] = (uint32_t)l[i].z;
        }
    }
    return TPM_OK;
}

int tpm_pm_export(tpm_ctx *h, tpm_sys sid, float *phi, int64_t count) {
    clear_error();
    if (!h || !phi) {
        set_error("null argument");
        return TPM_EINVAL;
    }
    Ctx *c = reinterpret_cast<Ctx *>(h);
    System *s = find(c, sid);
    if (!s) {
        set_error("unknown system handle %llu", (unsigned long long)sid);
        return TPM_ENOSYS_HANDLE;
    }
    if (!s->phi) {
        set_error("no long-range mesh: call tpm_pm_long_range first");
        return TPM_EINVAL;
    }
    const int64_t ncell = (int64_t)s->pm_mesh * s->pm_mesh * s->pm_mesh;
    if (count != ncell) {
        set_error("count must be the mesh size^3 = %lld", (long long)ncell);
        return TPM_EINVAL;
    }
    TPM_CUDA(cudaSetDevice(c->device));
    TPM_CUDA(cudaDeviceSynchronize());
    TPM_CUDA(cudaMemcpy(phi, s->phi, ncell * sizeof(float), cudaMemcpyDeviceToHost));
    return TPM_OK;
}

}  // extern "C"
