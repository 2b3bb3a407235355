// tpm_compute_forces_noalloc: force evaluation on an active subset that
// allocates no device memory.
//
// tpm_compute_forces draws its per-call scratch (the active set sorted into
// key order, and the sort's temporary storage) from the context's memory
// pool.  Some callers cannot let a library allocate device memory in the
// middle of their time-step loop: programs that have already handed the
// device memory to their own allocator, or that must not pay for an
// allocation (and the failure mode that comes with it) at every step.  This
// entry point keeps that scratch in one file-scope device array instead, of
// fixed size, which every GPU that loads the library holds until the process
// exits.  The caller still passes the inputs and outputs, all in device
// memory.
#include <cub/cub.cuh>

#include <mutex>

#include "tpm_internal.cuh"

namespace tpm {
namespace {

constexpr int64_t kMaxActive = TPM_NOALLOC_MAX_ACTIVE;
constexpr size_t kIdsBytes = (size_t)kMaxActive * sizeof(uint32_t);
// CUB radix-sort temporary storage.  The sort runs on double buffers (keys /
// values and their alternates, all in the scratch), so CUB needs only its
// histograms and look-back state here, not copies of the keys.
constexpr size_t kSortTempBytes = size_t(2) << 20;
constexpr size_t kRunsBytes = (size_t)kMaxActive * sizeof(uint2);  // runs of spread-out walk groups
constexpr size_t kScratchBytes = 4 * kIdsBytes + kSortTempBytes + kRunsBytes + 256;

// The shared scratch: keys, values, alternate keys, alternate values, the
// sort's temporary storage, the walk's run list and its count.  Host code
// must not pass this symbol to a
// kernel -- on the host it only names a stand-in; its device address comes
// from cudaGetSymbolAddress (see scratch_on_device).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_scratch on `device` (which must be current).  Looked up
// once per device; the first call on a device therefore calls
// cudaGetSymbolAddress, which loads the library's device code there.
int scratch_on_device(int device, unsigned char **out) {
    if (device < 0 || device >= kMaxDevices) {
        set_error("device %d out of range for the no-allocation scratch", device);
        return TPM_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress of the no-allocation scratch failed: %s", cudaGetErrorString(e));
            return TPM_ECUDA;
        }
        g_scratch_ptr[device] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_ptr[device]);
    return TPM_OK;
}

// Sort keys of the active set (sorted position of each id) and its slots, in
// the no-allocation scratch; an id out of range sets bit 0 of the system's
// status word (which tpm_sync_status reports) and is read as particle 0.
__global__ void k_noalloc_active_keys(const uint32_t *__restrict__ ids, int64_t n_act,
                                      const uint32_t *__restrict__ rank, int64_t n, uint32_t *__restrict__ keys,
                                      uint32_t *__restrict__ vals, int *__restrict__ err) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n_act)
        return;
    uint32_t id = ids[k];
    if (id >= (uint64_t)n) {
        atomicOr(err, 1);
        id = 0;
    }
    keys[k] = rank[id];
    vals[k] = (uint32_t)k;
}

// True for NULL, managed memory, and device memory of `device` (memory of
// another GPU would be dereferenced from the wrong device).
bool on_device(const void *p, int device) {
    if (!p)
        return true;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged)
        return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

}  // namespace
}  // namespace tpm

using namespace tpm;

extern "C" int tpm_compute_forces_noalloc(tpm_ctx *h, tpm_sys sid, const uint32_t *active_ids, int64_t n_active,
                                          const float *a_old, const tpm_force_params *p, float *acc, float *pot,
                                          uint32_t *n_int, void *stream) {
    clear_error();
    if (!h || !active_ids || !acc || !p) {
        set_error("null argument (active_ids, acc and params are required)");
        return TPM_EINVAL;
    }
    if (n_active < 1 || n_active > kMaxActive) {
        set_error("n_active = %lld outside [1, %lld], the fixed size of the no-allocation scratch",
                  (long long)n_active, (long long)kMaxActive);
        return TPM_EINVAL;
    }
    Ctx *c = reinterpret_cast<Ctx *>(h);
    System *s = nullptr;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        auto it = c->systems.find(sid);
        if (it != c->systems.end())
            s = it->second;
    }
    if (!s) {
        set_error("unknown system handle %llu", (unsigned long long)sid);
        return TPM_ENOSYS_HANDLE;
    }
    if (p->crit != TPM_CRIT_BH && p->crit != TPM_CRIT_RELATIVE) {
        set_error("crit must be TPM_CRIT_BH or TPM_CRIT_RELATIVE");
        return TPM_EINVAL;
    }
    if (p->crit == TPM_CRIT_RELATIVE && !a_old) {
        set_error("the relative criterion needs a_old");
        return TPM_EINVAL;
    }
    if (p->treepm && (!s->phi || s->pm_n != p->pm_n || s->pm_grad != p->pm_grad)) {
        set_error("no long-range mesh for these parameters: call tpm_pm_long_range first");
        return TPM_EINVAL;
    }
    TPM_CUDA(cudaSetDevice(c->device));
    const int dv = c->device;
    if (!on_device(active_ids, dv) || !on_device(a_old, dv) || !on_device(acc, dv) || !on_device(pot, dv) ||
        !on_device(n_int, dv)) {
        set_error("all arrays must be device memory of the context's GPU: host arrays would need staging buffers");
        return TPM_EINVAL;
    }
    unsigned char *base = nullptr;
    TPM_CHECK(scratch_on_device(c->device, &base));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    uint32_t *keys = reinterpret_cast<uint32_t *>(base);
    uint32_t *vals = reinterpret_cast<uint32_t *>(base + kIdsBytes);
    uint32_t *akeys = reinterpret_cast<uint32_t *>(base + 2 * kIdsBytes);
    uint32_t *avals = reinterpret_cast<uint32_t *>(base + 3 * kIdsBytes);
    void *sort_tmp = base + 4 * kIdsBytes;
    uint2 *runs = reinterpret_cast<uint2 *>(base + 4 * kIdsBytes + kSortTempBytes);
    unsigned *nruns = reinterpret_cast<unsigned *>(base + 4 * kIdsBytes + kSortTempBytes + kRunsBytes);

    int bits = 1;
    while ((int64_t(1) << bits) < s->n)
        bits++;
    // every buffer is written before it is read, so nothing in the shared
    // scratch needs clearing; the result ends in either half of each pair
    cub::DoubleBuffer<uint32_t> dk(keys, akeys), dvv(vals, avals);
    size_t need = 0;
    TPM_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, need, dk, dvv, (int)n_active, 0, bits, st));
    if (need > kSortTempBytes) {
        set_error("sort needs %zu bytes of temporary storage, the no-allocation scratch has %zu", need,
                  kSortTempBytes);
        return TPM_EINVAL;
    }
    k_noalloc_active_keys<<<(unsigned)((n_active + 255) / 256), 256, 0, st>>>(active_ids, n_active, s->rank, s->n,
                                                                             keys, vals, s->err);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    TPM_CUDA(cub::DeviceRadixSort::SortPairs(sort_tmp, need, dk, dvv, (int)n_active, 0, bits, st));
    count_cub_call();

    WalkRequest r{};
    r.sorted_idx = dk.Current();
    r.slot = dvv.Current();
    r.a_old = p->crit == TPM_CRIT_RELATIVE ? a_old : nullptr;
    r.n_act = n_active;
    r.acc = acc;
    r.pot = pot;
    r.nint = n_int;
    r.no_alloc = 1;
    r.runs = runs;    // the walk clears the count
    r.nruns = nruns;
    if (p->treepm) {
        TPM_CHECK(pm_interp_device(c, s, r, st));
        r.accumulate = 1;
    }
    return walk_device(c, s, p, r, st);
}
