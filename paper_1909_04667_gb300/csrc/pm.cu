// Periodic particle-mesh long-range force (paper Sec. 3.3, 3.4).
//
//   K6  cloud-in-cell assignment of every particle's mass to the 8 mesh points
//       around it (mesh points at x = i box / N), FP32 atomics
//   --  real-to-complex FFT (cuFFT)
//   K7  multiply by the Green's function of the long-range potential,
//       -4 pi G / k^2 exp(-k^2 r_s^2), divided by the square of the CIC window
//       W(k) = prod_a sinc^2(k_a dx / 2) (one window for assignment, one for
//       interpolation), with the k = 0 mode removed (the mean density does not
//       source the potential) and the inverse-FFT normalisation folded in.
//       The same pass also forms the three force spectra: the 4-point
//       finite difference dPhi/dx ~ [4/3 (Phi_{+1} - Phi_{-1})/2 -
//       1/3 (Phi_{+2} - Phi_{-2})/4] / dx is a circular convolution on the
//       periodic mesh, so it equals multiplication by its transfer function
//       i [4/3 sin(theta) - 1/6 sin(2 theta)] / dx, theta = 2 pi n / N.
//       Applying it in k-space gives the finite-difference force mesh without
//       the FP32 cancellation of differencing a smooth potential.
//   --  one batched complex-to-real FFT -> potential and 3 force meshes
//   K8  per active particle: CIC interpolation of force and potential
#include "tpm_internal.cuh"

namespace tpm {
namespace {

constexpr int kThreads = 256;
constexpr double kPi = 3.14159265358979323846;

__global__ void k_cic_deposit(const double *__restrict__ pos, const float *__restrict__ mass,
                              const uint32_t *__restrict__ perm, int64_t n, int ng, double cells_per_len,
                              float *__restrict__ rho) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n)
        return;
    const uint32_t j = perm[s];  // key order: neighbouring threads hit neighbouring cells
    int i0[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const double t = pos[3 * j + a] * cells_per_len;
        const double fl = floor(t);
        f[a] = (float)(t - fl);
        int q = (int)fl;
        q %= ng;
        if (q < 0)
            q += ng;
        i0[a] = q;
    }
    const float m = mass[j];
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        const float w = (dx ? f[0] : 1.0f - f[0]) * (dy ? f[1] : 1.0f - f[1]) * (dz ? f[2] : 1.0f - f[2]);
        int ix = i0[0] + dx, iy = i0[1] + dy, iz = i0[2] + dz;
        ix -= ix >= ng ? ng : 0;
        iy -= iy >= ng ? ng : 0;
        iz -= iz >= ng ? ng : 0;
        atomicAdd(&rho[((size_t)ix * ng + iy) * ng + iz], m * w);
    }
}

// sin(x)/x with the accurate sinf: the fast __sinf has an absolute error of
// ~4e-7, i.e. a relative error of ~3e-5 at the fundamental mode of a 256^3 mesh.
__device__ __forceinline__ float sinc_f(float x) { return x == 0.0f ? 1.0f : sinf(x) / x; }

// K7 on the r2c half spectrum [ng][ng][ng/2+1]: spec[0] (in place) becomes the
// potential spectrum, spec[1..3] the x, y, z force spectra.
__global__ void k_green(cufftComplex *__restrict__ spec, int64_t nspec, int ng, float kfund, float dx, float rs2,
                        float pref) {
    const int nzh = ng / 2 + 1;
    const float inv_dx = 1.0f / dx;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nspec;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int iz = (int)(e % nzh);
        const int iy = (int)((e / nzh) % ng);
        const int ix = (int)(e / ((int64_t)nzh * ng));
        const int n3[3] = {ix < ng / 2 ? ix : ix - ng, iy < ng / 2 ? iy : iy - ng, iz};
        float k2 = 0.0f, w = 1.0f, d[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const float ka = kfund * n3[a];
            k2 = fmaf(ka, ka, k2);
            w *= sinc_f(0.5f * ka * dx);
            const float th = 2.0f * (float)n3[a] / (float)ng;  // theta / pi
            d[a] = (4.0f / 3.0f * sinpif(th) - 1.0f / 6.0f * sinpif(2.0f * th)) * inv_dx;
        }
        cufftComplex v = spec[e];
        float g = 0.0f;
        if (k2 > 0.0f) {
            const float w2 = w * w;  // sinc^2 per axis
            g = pref * __expf(-k2 * rs2) / (k2 * w2 * w2);
        }
        const float re = v.x * g, im = v.y * g;
        spec[e] = make_float2(re, im);
        // force = -grad Phi: multiply by -i d
#pragma unroll
        for (int a = 0; a < 3; a++)
            spec[(a + 1) * nspec + e] = make_float2(d[a] * im, -d[a] * re);
    }
}

__device__ __forceinline__ int wrapi(int i, int ng) {
    i %= ng;
    return i < 0 ? i + ng : i;
}

// K8: CIC interpolation of the force meshes and the potential mesh.
__global__ void k_pm_interp(const float *__restrict__ mesh, int64_t ncell, int ng, double cells_per_len,
                            const double *__restrict__ pos, const uint32_t *__restrict__ perm,
                            const uint32_t *__restrict__ sidx, const uint32_t *__restrict__ slot, int64_t n_act,
                            float *__restrict__ acc, float *__restrict__ pot) {
    int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gi >= n_act)
        return;
    const uint32_t s = sidx ? sidx[gi] : (uint32_t)gi;
    const uint32_t out = slot ? slot[gi] : perm[s];
    const uint32_t j = perm[s];
    int i0[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const double t = pos[3 * j + a] * cells_per_len;
        const double fl = floor(t);
        f[a] = (float)(t - fl);
        i0[a] = wrapi((int)fl, ng);
    }
    float ph = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        const float w = (dx ? f[0] : 1.0f - f[0]) * (dy ? f[1] : 1.0f - f[1]) * (dz ? f[2] : 1.0f - f[2]);
        int x = i0[0] + dx, y = i0[1] + dy, z = i0[2] + dz;
        x -= x >= ng ? ng : 0;
        y -= y >= ng ? ng : 0;
        z -= z >= ng ? ng : 0;
        const size_t idx = ((size_t)x * ng + y) * ng + z;
        ph = fmaf(w, __ldg(&mesh[idx]), ph);
        gx = fmaf(w, __ldg(&mesh[ncell + idx]), gx);
        gy = fmaf(w, __ldg(&mesh[2 * ncell + idx]), gy);
        gz = fmaf(w, __ldg(&mesh[3 * ncell + idx]), gz);
    }
    acc[3 * (size_t)out] = gx;
    acc[3 * (size_t)out + 1] = gy;
    acc[3 * (size_t)out + 2] = gz;
    if (pot)
        pot[out] = ph;
}

}  // namespace

int pm_solve_device(Ctx *c, System *s, const tpm_force_params *p, cudaStream_t st) {
    const int ng = p->pm_n;
    const double box = s->bp.box;
    const double rs = p->asmth * box / ng;
    const int64_t ncell = (int64_t)ng * ng * ng;
    const int64_t nspec = (int64_t)ng * ng * (ng / 2 + 1);

    // plans are cached per mesh size
    cufftHandle fwd, inv;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        auto it = c->fft_plans.find(ng);
        if (it == c->fft_plans.end()) {
            if (cufftPlan3d(&fwd, ng, ng, ng, CUFFT_R2C) != CUFFT_SUCCESS) {
                set_error("cufftPlan3d (R2C, %d^3) failed", ng);
                return TPM_ECUDA;
            }
            int dims[3] = {ng, ng, ng};
            if (cufftPlanMany(&inv, 3, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_C2R, 4) != CUFFT_SUCCESS) {
                cufftDestroy(fwd);
                set_error("cufftPlanMany (C2R x 4, %d^3) failed", ng);
                return TPM_ECUDA;
            }
            c->fft_plans[ng] = {fwd, inv};
        } else {
            fwd = it->second.first;
            inv = it->second.second;
        }
    }
    if (s->pm_n != ng) {
        s->pm_mem.release(st);
        s->phi = nullptr;
        s->pm_mem.ctx = c;
        TPM_CHECK(s->pm_mem.get(&s->phi, 4 * ncell, st));  // potential, then x, y, z force
        s->pm_n = ng;
    }
    AllocSet tmp;
    tmp.ctx = c;
    struct Guard {
        AllocSet &t;
        cudaStream_t st;
        ~Guard() { t.release(st); }
    } guard{tmp, st};
    cufftComplex *spec;
    TPM_CHECK(tmp.get(&spec, 4 * nspec, st));
    float *rho = s->phi;  // the density occupies the potential slot until the inverse FFT
    TPM_CUDA(cudaMemsetAsync(rho, 0, ncell * sizeof(float), st));
    const double cpl = ng / box;
    k_cic_deposit<<<(unsigned)((s->n + kThreads - 1) / kThreads), kThreads, 0, st>>>(s->pos, s->mass, s->perm, s->n,
                                                                                     ng, cpl, rho);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    if (cufftSetStream(fwd, st) != CUFFT_SUCCESS || cufftExecR2C(fwd, rho, spec) != CUFFT_SUCCESS) {
        set_error("cufftExecR2C failed");
        return TPM_ECUDA;
    }
    const double dx = box / ng;
    // density = mass / dx^3; inverse FFT normalisation 1 / ng^3
    const double pref = -4.0 * kPi * s->bp.G / (dx * dx * dx) / (double)ncell;
    k_green<<<(unsigned)(c->num_sms * 8), kThreads, 0, st>>>(spec, nspec, ng, (float)(2.0 * kPi / box), (float)dx,
                                                            (float)(rs * rs), (float)pref);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    if (cufftSetStream(inv, st) != CUFFT_SUCCESS || cufftExecC2R(inv, spec, s->phi) != CUFFT_SUCCESS) {
        set_error("cufftExecC2R failed");
        return TPM_ECUDA;
    }
    s->pm_rs = rs;
    s->pm_G = s->bp.G;
    return TPM_OK;
}

int pm_interp_device(Ctx *, const System *s, const WalkRequest &r, cudaStream_t st) {
    if (r.n_act == 0)
        return TPM_OK;
    const int ng = s->pm_n;
    const double box = s->bp.box;
    k_pm_interp<<<(unsigned)((r.n_act + kThreads - 1) / kThreads), kThreads, 0, st>>>(
        s->phi, (int64_t)ng * ng * ng, ng, ng / box, s->pos, s->perm, r.sorted_idx, r.slot, r.n_act, r.acc, r.pot);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    return TPM_OK;
}

}  // namespace tpm
