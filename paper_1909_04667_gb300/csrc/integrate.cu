// Time stepping around the force path (paper Sec. 7.1-7.3): drift, the set of
// particles due at a tick of the power-of-two hierarchy, and the closing /
// opening half kicks with the re-binning between them.
//
// Bins: bin b (0 <= b <= N = nbins - 1) has the step dt_tick 2^(N - b), so
// bin 0 is the longest step and bin N the shortest; bin b is due at tick t
// when t is a multiple of 2^(N - b).  Every FP64 update below uses explicit
// round-to-nearest multiplies and adds in a fixed order (no contraction), so
// the same forces give the same bits on any correct implementation.
#include <cub/cub.cuh>
#include <thrust/iterator/counting_iterator.h>

#include <cmath>

#include "tpm_internal.cuh"

namespace tpm {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxBins = 31;

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

bool device_ptr(const void *p) {
    if (!p)
        return false;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// x += v dt over the 3n coordinates; periodic coordinates are wrapped back
// into [0, box) by x - floor(x / box) box (and one more box if rounding left
// x == box).
__global__ void k_drift(double *__restrict__ x, const double *__restrict__ v, int64_t m, double dt, int periodic,
                        double box) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += stride) {
        double y = __dadd_rn(x[i], __dmul_rn(v[i], dt));
        if (periodic) {
            y = __dsub_rn(y, __dmul_rn(floor(__ddiv_rn(y, box)), box));
            if (y >= box)
                y = __dsub_rn(y, box);
        }
        x[i] = y;
    }
}

struct DueAt {
    const int8_t *bins;
    int64_t tick;
    int top;  // N
    __device__ __forceinline__ bool operator()(uint32_t i) const {
        const int b = min(max((int)bins[i], 0), top);
        return (tick & ((int64_t(1) << (top - b)) - 1)) == 0;
    }
};

// |a| of the selected particles' last force, in selection order (the relative
// criterion's a_old for the coming force call).
__global__ void k_gather_amag(const uint32_t *__restrict__ ids, const int *__restrict__ n_sel,
                              const float *__restrict__ amag, float *__restrict__ out) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < *n_sel)
        out[k] = amag[ids[k]];
}

// Step of bin b: dt_tick 2^(N - b) (exact: a power-of-two scaling).
__device__ __forceinline__ double bin_step(double dt_tick, int top, int b) { return ldexp(dt_tick, top - b); }

// Closing half kick with the step that ends (unless `first`), the new bin --
// the largest step not above sqrt(2 C_grav eps / |a|), moved towards the old
// bin until it is due at `tick` when it is longer than the old one -- and the
// opening half kick with the new step.  |a| (FP64 from the FP32 force) is
// kept for the next evaluation's relative criterion.
__global__ void k_kick(const uint32_t *__restrict__ ids, int64_t n_act, int64_t n, const float *__restrict__ acc,
                       double *__restrict__ vel, int8_t *__restrict__ bins, float *__restrict__ amag, int64_t tick,
                       double dt_tick, int top, double two_c_eps, int first) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n_act)
        return;
    const uint32_t i = ids[k];
    if (i >= n)
        return;  // not a particle: skipped
    const double a[3] = {(double)acc[3 * k], (double)acc[3 * k + 1], (double)acc[3 * k + 2]};
    double v[3] = {vel[3 * (size_t)i], vel[3 * (size_t)i + 1], vel[3 * (size_t)i + 2]};
    const int b_old = min(max((int)bins[i], 0), top);
    if (!first) {
        const double h = bin_step(dt_tick, top, b_old);
        for (int c = 0; c < 3; c++)
            v[c] = __dadd_rn(v[c], __dmul_rn(__dmul_rn(a[c], h), 0.5));
    }
    const double am = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(a[0], a[0]), __dmul_rn(a[1], a[1])), __dmul_rn(a[2], a[2])));
    const double dt_max = am > 0.0 ? sqrt(__ddiv_rn(two_c_eps, am)) : INFINITY;
    int b = top;
    for (int c = 0; c <= top; c++)
        if (bin_step(dt_tick, top, c) <= dt_max) {
            b = c;
            break;
        }
    if (!first && b < b_old)
        while (b < top && (tick & ((int64_t(1) << (top - b)) - 1)) != 0)
            b++;  // ends at b_old at the latest: it is due now
    const double h = bin_step(dt_tick, top, b);
    for (int c = 0; c < 3; c++)
        v[c] = __dadd_rn(v[c], __dmul_rn(__dmul_rn(a[c], h), 0.5));
    vel[3 * (size_t)i] = v[0];
    vel[3 * (size_t)i + 1] = v[1];
    vel[3 * (size_t)i + 2] = v[2];
    bins[i] = (int8_t)b;
    amag[i] = (float)am;
}

}  // namespace
}  // namespace tpm

using namespace tpm;

extern "C" int tpm_drift(tpm_ctx *h, double *pos, const double *vel, int64_t n, double dt, int32_t periodic,
                         double box, void *stream) {
    clear_error();
    if (!h || n < 0 || (n > 0 && (!pos || !vel)) || !std::isfinite(dt) || (periodic && !(box > 0.0))) {
        set_error("tpm_drift: null argument, n < 0, non-finite dt or box <= 0");
        return TPM_EINVAL;
    }
    if (n == 0)
        return TPM_OK;
    Ctx *c = reinterpret_cast<Ctx *>(h);
    TPM_CUDA(cudaSetDevice(c->device));
    if (!device_ptr(pos) || !device_ptr(vel)) {
        set_error("tpm_drift: pos and vel must be device memory");
        return TPM_EINVAL;
    }
    const int64_t m = 3 * n;
    const unsigned grid = (unsigned)std::min<int64_t>(blocks_for(m), (int64_t)c->num_sms * 8);
    k_drift<<<grid, kThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(pos, vel, m, dt, periodic ? 1 : 0, box);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    return TPM_OK;
}

extern "C" int tpm_active_set(tpm_ctx *h, const int8_t *bins, const float *amag, int64_t n, int64_t tick,
                              int32_t nbins, uint32_t *ids, float *a_old, int64_t *n_active, void *stream) {
    clear_error();
    if (!h || !bins || !ids || !n_active || n < 1 || n > 0x7fffffffLL || nbins < 1 || nbins > kMaxBins ||
        tick < 0 || (a_old && !amag)) {
        set_error("tpm_active_set: null argument, n outside [1, 2^31 - 1], nbins outside [1, %d] or tick < 0",
                  kMaxBins);
        return TPM_EINVAL;
    }
    Ctx *c = reinterpret_cast<Ctx *>(h);
    TPM_CUDA(cudaSetDevice(c->device));
    if (!device_ptr(bins) || !device_ptr(ids) || (a_old && (!device_ptr(a_old) || !device_ptr(amag)))) {
        set_error("tpm_active_set: bins, ids, amag and a_old must be device memory");
        return TPM_EINVAL;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int top = nbins - 1;
    const int64_t t = tick & ((int64_t(1) << top) - 1);  // position in the cycle
    DueAt pred{bins, t, top};
    thrust::counting_iterator<uint32_t> it(0);
    AllocSet tmp;
    tmp.ctx = c;
    struct Guard {
        AllocSet &a;
        cudaStream_t st;
        ~Guard() { a.release(st); }
    } guard{tmp, st};
    int *n_sel;
    TPM_CHECK(tmp.get(&n_sel, 1, st));
    size_t bytes = 0;
    TPM_CUDA(cub::DeviceSelect::If(nullptr, bytes, it, ids, n_sel, (int)n, pred, st));
    char *scratch;
    TPM_CHECK(tmp.get(&scratch, bytes, st));
    TPM_CUDA(cub::DeviceSelect::If(scratch, bytes, it, ids, n_sel, (int)n, pred, st));
    count_cub_call();
    if (a_old) {
        k_gather_amag<<<blocks_for(n), kThreads, 0, st>>>(ids, n_sel, amag, a_old);
        count_launch();
        TPM_CUDA(cudaGetLastError());
    }
    int host_n = 0;
    TPM_CUDA(cudaMemcpyAsync(&host_n, n_sel, sizeof(int), cudaMemcpyDeviceToHost, st));
    TPM_CUDA(cudaStreamSynchronize(st));
    *n_active = host_n;
    return TPM_OK;
}

extern "C" int tpm_kick(tpm_ctx *h, const uint32_t *ids, int64_t n_active, int64_t n, const float *acc,
                        double *vel, int8_t *bins, float *amag, int64_t tick, const tpm_step_params *p,
                        int32_t first, void *stream) {
    clear_error();
    if (!h || !p || n_active < 0 || n < 0 || (n_active > 0 && (!ids || !acc || !vel || !bins || !amag))) {
        set_error("tpm_kick: null argument, n_active < 0 or n < 0");
        return TPM_EINVAL;
    }
    if (p->nbins < 1 || p->nbins > kMaxBins || !(p->dt_tick > 0.0) || !std::isfinite(p->dt_tick) ||
        !(p->c_grav > 0.0) || !(p->eps > 0.0) || tick < 0) {
        set_error("tpm_kick: nbins outside [1, %d], or dt_tick, c_grav, eps not > 0, or tick < 0", kMaxBins);
        return TPM_EINVAL;
    }
    if (n_active == 0)
        return TPM_OK;
    Ctx *c = reinterpret_cast<Ctx *>(h);
    TPM_CUDA(cudaSetDevice(c->device));
    if (!device_ptr(ids) || !device_ptr(acc) || !device_ptr(vel) || !device_ptr(bins) || !device_ptr(amag)) {
        set_error("tpm_kick: all arrays must be device memory");
        return TPM_EINVAL;
    }
    const int top = p->nbins - 1;
    const int64_t t = tick & ((int64_t(1) << top) - 1);
    const double two_c_eps = 2.0 * p->c_grav * p->eps;
    k_kick<<<blocks_for(n_active), kThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        ids, n_active, n, acc, vel, bins, amag, t, p->dt_tick, top, two_c_eps, first ? 1 : 0);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    return TPM_OK;
}
