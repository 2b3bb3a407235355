// Batched force evaluation: many active-set requests, on one or several
// resident trees, in one persistent walk launch.
//
// With local power-of-two time steps (paper Sec. 7.2) most substeps activate
// only a small fraction of the particles, and a force server sees many small
// requests for different systems.  Launching one walk per request pays a
// launch, a sort and a tail of idle SMs each time.  Here a plan holds all the
// scratch a batch needs (allocated once), so a batched call only enqueues
// kernels -- no allocation, no host synchronisation -- and a sequence of
// batched calls can be captured in a CUDA graph.  Per call:
//   1. each request's ids are mapped to positions in its tree's key order
//      (and, unless the caller says they already are, sorted by (request,
//      key order)),
//   2. each request is cut into groups of at most G consecutive particles
//      (G is the plan's group size, chosen by tpm_plan_autotune),
//   3. one persistent walk launch lets resident warps take groups from a
//      device work queue until it is empty.
#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "tpm_internal.cuh"

namespace tpm {
namespace {

struct KeyReq {
    const uint32_t *rank;
    int64_t n;
};

struct Plan {
    Ctx *ctx = nullptr;
    int64_t max_ids = 0, max_req = 0, max_groups = 0;
    int group_size = 32;
    int stack_depth = 192;  // candidate-stack capacity of the batched walk
    AllocSet mem;
    uint64_t *keys = nullptr, *skeys = nullptr;
    uint32_t *vals = nullptr, *slot = nullptr, *sidx = nullptr;
    uint32_t *gcnt = nullptr, *goff = nullptr;
    uint4 *groups = nullptr;
    unsigned *ngroups = nullptr, *next = nullptr;
    int *err = nullptr;
    int64_t *off_dev = nullptr;
    KeyReq *kreq_dev = nullptr;
    unsigned char *reqs_dev = nullptr;
    int64_t *off_host = nullptr;
    KeyReq *kreq_host = nullptr;
    unsigned char *reqs_host = nullptr;
    void *cub_tmp = nullptr;
    size_t cub_bytes = 0;
    cudaEvent_t staged = nullptr;  // host staging buffers may be rewritten once this has passed
    bool staged_pending = false;
};

// Per requested id (one thread each, over all requests: one block per
// request left a large request to a single block): the sorted position of the
// id in its own tree; either directly the walk's sorted index (requests given
// in key order) or a (request, sorted position) sort key with the id's slot.
// The request of position i is the last r with off[r] <= i (empty requests
// share their offset with the next one).  An id out of range sets bit 0 of
// the status word and is read as particle 0.
__global__ void k_batch_keys(const KeyReq *__restrict__ kr, const int64_t *__restrict__ off, int64_t n_req,
                             int64_t n_ids, const uint32_t *__restrict__ ids, int presorted,
                             uint64_t *__restrict__ keys, uint32_t *__restrict__ vals, uint32_t *__restrict__ sidx,
                             uint32_t *__restrict__ slot, int *__restrict__ err) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_ids)
        return;
    int64_t lo = 0, hi = n_req - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    const int64_t r = lo;
    uint32_t id = ids[i];
    if (id >= (uint64_t)kr[r].n) {
        atomicOr(err, 1);
        id = 0;
    }
    const uint32_t rk = kr[r].rank[id];
    if (presorted) {
        sidx[i] = rk;
        slot[i] = (uint32_t)i;
    } else {
        keys[i] = ((uint64_t)r << 32) | rk;
        vals[i] = (uint32_t)i;
    }
}

// Sorted (request, position) keys back to sorted positions.
__global__ void k_batch_unpack(const uint64_t *__restrict__ skeys, int64_t n, uint32_t *__restrict__ sidx) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n)
        sidx[i] = (uint32_t)skeys[i];
}

// Number of walk groups of at most g particles per request.
__global__ void k_batch_gcount(const int64_t *__restrict__ off, int64_t n_req, int g, uint32_t *__restrict__ gcnt) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < n_req)
        gcnt[r] = (uint32_t)((off[r + 1] - off[r] + g - 1) / g);
}

// The group table of the persistent walk: (start, count, request, 0) for each
// group of each request, from the scanned group counts; the total into ngroups.
__global__ void k_batch_groups(const int64_t *__restrict__ off, const uint32_t *__restrict__ gcnt,
                               const uint32_t *__restrict__ goff, int64_t n_req, int g, uint4 *__restrict__ groups,
                               unsigned *__restrict__ ngroups) {
    const int64_t r = blockIdx.x;
    const int64_t lo = off[r], hi = off[r + 1];
    const uint32_t base = goff[r], ng = gcnt[r];
    for (uint32_t q = threadIdx.x; q < ng; q += blockDim.x) {
        const int64_t start = lo + (int64_t)q * g;
        groups[base + q] = make_uint4((uint32_t)start, (uint32_t)min((int64_t)g, hi - start), (uint32_t)r, 0u);
    }
    if (r == n_req - 1 && threadIdx.x == 0)
        *ngroups = base + ng;
}

int end_bit_for(int64_t n_req) {
    int b = 1;
    while ((int64_t(1) << b) < n_req)
        b++;
    return 32 + b;
}

bool dev_ptr(const void *p) {
    if (!p)
        return true;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Frees a plan's device and host memory (not the Plan object itself).
void release_plan(Plan *pl) {
    cudaDeviceSynchronize();
    pl->mem.release(0);
    cudaStreamSynchronize(0);
    if (pl->off_host)
        cudaFreeHost(pl->off_host);
    if (pl->kreq_host)
        cudaFreeHost(pl->kreq_host);
    if (pl->reqs_host)
        cudaFreeHost(pl->reqs_host);
    if (pl->staged)
        cudaEventDestroy(pl->staged);
    pl->off_host = nullptr;
    pl->kreq_host = nullptr;
    pl->reqs_host = nullptr;
    pl->staged = nullptr;
}

int run_batch(Ctx *c, Plan *pl, int64_t n_req, const tpm_sys *systems, const int64_t *offsets,
              const tpm_force_params *params, const uint32_t *ids, const float *a_old, float *acc, float *pot,
              uint32_t *nint, uint32_t flags, cudaStream_t st) {
    if (n_req < 1 || n_req > pl->max_req) {
        set_error("n_req = %lld outside [1, %lld] (plan size)", (long long)n_req, (long long)pl->max_req);
        return TPM_EINVAL;
    }
    if (!systems || !offsets || !params || !ids || !acc) {
        set_error("null argument");
        return TPM_EINVAL;
    }
    if (offsets[0] != 0) {
        set_error("offsets[0] must be 0");
        return TPM_EINVAL;
    }
    for (int64_t r = 0; r < n_req; r++)
        if (offsets[r + 1] < offsets[r]) {
            set_error("offsets must not decrease");
            return TPM_EINVAL;
        }
    const int64_t n_ids = offsets[n_req];
    if (n_ids > pl->max_ids) {
        set_error("%lld ids exceed the plan's %lld", (long long)n_ids, (long long)pl->max_ids);
        return TPM_EINVAL;
    }
    if (!dev_ptr(ids) || !dev_ptr(a_old) || !dev_ptr(acc) || !dev_ptr(pot) || !dev_ptr(nint)) {
        set_error("batched evaluation takes device arrays only");
        return TPM_EINVAL;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    TPM_CUDA(cudaStreamIsCapturing(st, &cap));
    // the host staging buffers of the previous call must have been copied
    if (pl->staged_pending && cap == cudaStreamCaptureStatusNone) {
        TPM_CUDA(cudaEventSynchronize(pl->staged));
        pl->staged_pending = false;
    }
    const size_t rb = batch_req_bytes();
    {
        std::lock_guard<std::mutex> lk(c->mu);
        for (int64_t r = 0; r < n_req; r++) {
            auto it = c->systems.find(systems[r]);
            if (it == c->systems.end()) {
                set_error("unknown system handle %llu in request %lld", (unsigned long long)systems[r], (long long)r);
                return TPM_ENOSYS_HANDLE;
            }
            const System *s = it->second;
            const tpm_force_params *p = &params[r];
            if (s->bp.periodic || p->treepm || s->psoft) {
                set_error("batched evaluation supports open boundaries with uniform softening (request %lld)", (long long)r);
                return TPM_EINVAL;
            }
            if (p->crit != TPM_CRIT_BH && p->crit != TPM_CRIT_RELATIVE) {
                set_error("bad criterion in request %lld", (long long)r);
                return TPM_EINVAL;
            }
            if (p->crit == TPM_CRIT_RELATIVE && !a_old) {
                set_error("request %lld uses the relative criterion: a_old is required", (long long)r);
                return TPM_EINVAL;
            }
            pl->kreq_host[r] = KeyReq{s->rank, s->n};
            fill_batch_req(pl->reqs_host + r * rb, s, p);
            pl->off_host[r] = offsets[r];
        }
        pl->off_host[n_req] = n_ids;
    }
    if (n_ids == 0)
        return TPM_OK;
    TPM_CUDA(cudaMemcpyAsync(pl->off_dev, pl->off_host, (n_req + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    TPM_CUDA(cudaMemcpyAsync(pl->kreq_dev, pl->kreq_host, n_req * sizeof(KeyReq), cudaMemcpyHostToDevice, st));
    TPM_CUDA(cudaMemcpyAsync(pl->reqs_dev, pl->reqs_host, n_req * rb, cudaMemcpyHostToDevice, st));
    if (cap == cudaStreamCaptureStatusNone) {
        TPM_CUDA(cudaEventRecord(pl->staged, st));
        pl->staged_pending = true;
    }
    const bool presorted = flags & TPM_BATCH_PRESORTED;
    k_batch_keys<<<(unsigned)((n_ids + 255) / 256), 256, 0, st>>>(pl->kreq_dev, pl->off_dev, n_req, n_ids, ids,
                                                                  presorted ? 1 : 0, pl->keys, pl->vals, pl->sidx,
                                                                  pl->slot, pl->err);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    if (!presorted) {
        size_t b = pl->cub_bytes;
        TPM_CUDA(cub::DeviceRadixSort::SortPairs(pl->cub_tmp, b, pl->keys, pl->skeys, pl->vals, pl->slot, (int)n_ids,
                                                 0, end_bit_for(n_req), st));
        count_cub_call();
        k_batch_unpack<<<(unsigned)((n_ids + 255) / 256), 256, 0, st>>>(pl->skeys, n_ids, pl->sidx);
        count_launch();
    }
    const int g = pl->group_size;
    k_batch_gcount<<<(unsigned)((n_req + 255) / 256), 256, 0, st>>>(pl->off_dev, n_req, g, pl->gcnt);
    count_launch();
    size_t b = pl->cub_bytes;
    TPM_CUDA(cub::DeviceScan::ExclusiveSum(pl->cub_tmp, b, pl->gcnt, pl->goff, (int)n_req, st));
    count_cub_call();
    k_batch_groups<<<(unsigned)n_req, 128, 0, st>>>(pl->off_dev, pl->gcnt, pl->goff, n_req, g, pl->groups,
                                                    pl->ngroups);
    count_launch();
    TPM_CUDA(cudaMemsetAsync(pl->next, 0, sizeof(unsigned), st));
    TPM_CUDA(cudaGetLastError());
    return launch_walk_batch(c, g, pl->stack_depth, pl->reqs_dev, pl->groups, pl->ngroups, pl->next, pl->sidx,
                             pl->slot, a_old, acc, pot, nint, pl->err, st);
}

}  // namespace
}  // namespace tpm

using namespace tpm;

struct tpm_plan {
    Plan p;
};

extern "C" {

int tpm_plan_create(tpm_ctx *h, int64_t max_ids, int64_t max_requests, tpm_plan **out) {
    clear_error();
    if (!h || !out || max_ids < 1 || max_requests < 1 || max_ids > 0x7fffffffLL || max_requests > 0x7fffffffLL) {
        set_error("bad arguments: max_ids and max_requests must lie in [1, 2^31 - 1]");
        return TPM_EINVAL;
    }
    *out = nullptr;
    Ctx *c = reinterpret_cast<Ctx *>(h);
    TPM_CUDA(cudaSetDevice(c->device));
    tpm_plan *wrap = new tpm_plan;
    Plan *pl = &wrap->p;
    pl->ctx = c;
    pl->mem.ctx = c;
    pl->max_ids = max_ids;
    pl->max_req = max_requests;
    pl->max_groups = max_ids / 8 + max_requests + 1;  // group size >= 8
    const size_t rb = batch_req_bytes();
    int rc = TPM_OK;
    cudaStream_t st = 0;
    auto fail = [&](int code) {
        release_plan(pl);
        delete wrap;
        return code;
    };
    if ((rc = pl->mem.get(&pl->keys, max_ids, st)) || (rc = pl->mem.get(&pl->skeys, max_ids, st)) ||
        (rc = pl->mem.get(&pl->vals, max_ids, st)) || (rc = pl->mem.get(&pl->slot, max_ids, st)) ||
        (rc = pl->mem.get(&pl->sidx, max_ids, st)) || (rc = pl->mem.get(&pl->gcnt, max_requests, st)) ||
        (rc = pl->mem.get(&pl->goff, max_requests, st)) || (rc = pl->mem.get(&pl->groups, pl->max_groups, st)) ||
        (rc = pl->mem.get(&pl->ngroups, 1, st)) || (rc = pl->mem.get(&pl->next, 1, st)) ||
        (rc = pl->mem.get(&pl->err, 1, st)) || (rc = pl->mem.get(&pl->off_dev, max_requests + 1, st)) ||
        (rc = pl->mem.get(&pl->kreq_dev, max_requests, st)) ||
        (rc = pl->mem.get(&pl->reqs_dev, max_requests * rb, st)))
        return fail(rc);
    size_t sort_b = 0, scan_b = 0;
    if (cub::DeviceRadixSort::SortPairs(nullptr, sort_b, pl->keys, pl->skeys, pl->vals, pl->slot, (int)max_ids, 0,
                                        end_bit_for(max_requests), st) != cudaSuccess ||
        cub::DeviceScan::ExclusiveSum(nullptr, scan_b, pl->gcnt, pl->goff, (int)max_requests, st) != cudaSuccess) {
        set_error("CUB size query failed");
        return fail(TPM_ECUDA);
    }
    pl->cub_bytes = std::max(sort_b, scan_b);
    if ((rc = pl->mem.get((char **)&pl->cub_tmp, pl->cub_bytes, st)))
        return fail(rc);
    if (cudaMallocHost(&pl->off_host, (max_requests + 1) * sizeof(int64_t)) != cudaSuccess ||
        cudaMallocHost(&pl->kreq_host, max_requests * sizeof(KeyReq)) != cudaSuccess ||
        cudaMallocHost(&pl->reqs_host, max_requests * rb) != cudaSuccess ||
        cudaEventCreateWithFlags(&pl->staged, cudaEventDisableTiming) != cudaSuccess) {
        set_error("pinned staging allocation failed");
        return fail(TPM_ECUDA);
    }
    if (cudaMemsetAsync(pl->err, 0, sizeof(int), st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("plan initialisation failed");
        return fail(TPM_ECUDA);
    }
    *out = wrap;
    return TPM_OK;
}

int tpm_plan_destroy(tpm_ctx *h, tpm_plan *plan) {
    clear_error();
    if (!plan)
        return TPM_OK;
    if (!h) {
        set_error("null ctx");
        return TPM_EINVAL;
    }
    Ctx *c = reinterpret_cast<Ctx *>(h);
    cudaSetDevice(c->device);
    release_plan(&plan->p);
    delete plan;
    return TPM_OK;
}

int tpm_plan_set_group_size(tpm_plan *plan, int group_size) {
    clear_error();
    if (!plan || ((group_size < 8 || group_size > 32) && group_size != 64)) {
        set_error("group size must lie in [8, 32] or be 64");
        return TPM_EINVAL;
    }
    plan->p.group_size = group_size;
    return TPM_OK;
}

int tpm_plan_group_size(const tpm_plan *plan) { return plan ? plan->p.group_size : 0; }

int tpm_plan_set_stack_depth(tpm_plan *plan, int depth) {
    clear_error();
    if (!plan || (depth != 128 && depth != 192 && depth != 256)) {
        set_error("stack depth must be 128, 192 or 256");
        return TPM_EINVAL;
    }
    plan->p.stack_depth = depth;
    return TPM_OK;
}

int tpm_plan_stack_depth(const tpm_plan *plan) { return plan ? plan->p.stack_depth : 0; }

int tpm_compute_forces_batch(tpm_ctx *h, tpm_plan *plan, int64_t n_req, const tpm_sys *systems,
                             const int64_t *offsets, const tpm_force_params *params, const uint32_t *ids,
                             const float *a_old, float *acc, float *pot, uint32_t *n_int, uint32_t flags,
                             void *stream) {
    clear_error();
    if (!h || !plan) {
        set_error("null ctx or plan");
        return TPM_EINVAL;
    }
    Ctx *c = reinterpret_cast<Ctx *>(h);
    if (plan->p.ctx != c) {
        set_error("plan belongs to another context");
        return TPM_EINVAL;
    }
    TPM_CUDA(cudaSetDevice(c->device));
    return run_batch(c, &plan->p, n_req, systems, offsets, params, ids, a_old, acc, pot, n_int, flags,
                     reinterpret_cast<cudaStream_t>(stream));
}

int tpm_plan_sync_status(tpm_ctx *h, tpm_plan *plan, void *stream) {
    clear_error();
    if (!h || !plan) {
        set_error("null ctx or plan");
        return TPM_EINVAL;
    }
    Ctx *c = reinterpret_cast<Ctx *>(h);
    TPM_CUDA(cudaSetDevice(c->device));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int word = 0;
    TPM_CUDA(cudaMemcpyAsync(&word, plan->p.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    TPM_CUDA(cudaStreamSynchronize(st));
    if (!word)
        return TPM_OK;
    TPM_CUDA(cudaMemsetAsync(plan->p.err, 0, sizeof(int), st));
    TPM_CUDA(cudaStreamSynchronize(st));
    if (word & 1) {
        set_error("an id was out of range for its system (its outputs are those of particle 0)");
        return TPM_EINVAL;
    }
    set_error("the walk's candidate stack overflowed (device status %d)", word);
    return TPM_ECUDA;
}

int tpm_plan_autotune(tpm_ctx *h, tpm_plan *plan, int64_t n_req, const tpm_sys *systems, const int64_t *offsets,
                      const tpm_force_params *params, const uint32_t *ids, const float *a_old, float *acc,
                      float *pot, uint32_t *n_int, uint32_t flags, int reps, void *stream, int *best_group,
                      float *best_ms) {
    clear_error();
    if (!h || !plan || reps < 1) {
        set_error("null ctx or plan, or reps < 1");
        return TPM_EINVAL;
    }
    Ctx *c = reinterpret_cast<Ctx *>(h);
    TPM_CUDA(cudaSetDevice(c->device));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    TPM_CUDA(cudaEventCreate(&e0));
    TPM_CUDA(cudaEventCreate(&e1));
    const int groups[4] = {8, 16, 32, 64}, depths[3] = {128, 192, 256};
    int best = plan->p.group_size, best_depth = plan->p.stack_depth;
    float best_t = 1e30f;
    int rc = TPM_OK;
    for (int cand = 0; cand < 12 && rc == TPM_OK; cand++) {
        const int g = groups[cand / 3];
        plan->p.group_size = g;
        plan->p.stack_depth = depths[cand % 3];
        rc = run_batch(c, &plan->p, n_req, systems, offsets, params, ids, a_old, acc, pot, n_int, flags, st);
        if (rc != TPM_OK)
            break;
        std::vector<float> t;
        for (int r = 0; r < reps && rc == TPM_OK; r++) {
            cudaEventRecord(e0, st);
            rc = run_batch(c, &plan->p, n_req, systems, offsets, params, ids, a_old, acc, pot, n_int, flags, st);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                set_error("timing failed");
                rc = TPM_ECUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            t.push_back(ms);
        }
        if (rc != TPM_OK)
            break;
        std::sort(t.begin(), t.end());
        const float med = t[t.size() / 2];
        if (med < best_t) {
            best_t = med;
            best = g;
            best_depth = plan->p.stack_depth;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    plan->p.group_size = best;
    plan->p.stack_depth = best_depth;
    if (best_group)
        *best_group = best;
    if (best_ms)
        *best_ms = best_t;
    return rc;
}

}  // extern "C"
