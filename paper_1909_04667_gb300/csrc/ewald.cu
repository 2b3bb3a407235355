// Ewald correction of the periodic tree without the mesh (paper Sec. 3.1: the
// contributions of the mirrored images summed by the Ewald technique).
//
// For a unit mass (G = 1) at nearest-image separation d = x_source - x_target
// in a cube of side L with the mean density subtracted, the periodic
// acceleration of the target and its potential are, with the split a = 2 / L,
//   a_E(d)   = sum_n (d + nL)/s^3 [erfc(a s) + 2 a s / sqrt(pi) e^{-a^2 s^2}]
//              + (4 pi / V) sum_{k != 0} k / k^2 e^{-k^2 / 4a^2} sin(k.d)
//   phi_E(d) = -sum_n erfc(a s) / s - (4 pi / V) sum_{k != 0} e^{-k^2/4a^2} / k^2
//              cos(k.d) + pi / (a^2 V),
// s = |d + nL|, k = 2 pi m / L.  The walk adds the nearest image itself
// (spline-softened); the table holds what it misses, a_E - d / |d|^3 and
// phi_E + 1 / |d| (at d = 0: zero force and the particle's own lattice
// potential), on the grid d = (i, j, k) L / (2 kEwaldN), 0 <= i, j, k <=
// kEwaldN, as float4 (fx, fy, fz, phi) for unit box (it scales as 1 / L^2 and
// 1 / L).  Images |n| <= 3 (erfc(5) ~ 1.5e-12) and |m|^2 <= 30 (e^{-pi^2 m^2/4}
// < 1e-32).  Built in FP64 once per context and kept.
#include <cmath>

#include "tpm_internal.cuh"

namespace tpm {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kKmax = 5;
constexpr int kKw = 2 * kKmax + 1;

__constant__ double c_kweight[kKw * kKw * kKw];  // (4 pi / V) e^{-k^2/4a^2} / k^2 at unit box, 0 outside

__global__ void k_ewald_table(float4 *__restrict__ tab, int nt) {
    const int m = nt + 1;
    const int64_t total = (int64_t)m * m * m;
    const double a = 2.0, a2 = 4.0, sqpi = sqrt(kPi), tw = 2.0 * kPi;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / ((int64_t)m * m)), j = (int)((e / m) % m), l = (int)(e % m);
        const double step = 0.5 / nt;
        const double d[3] = {i * step, j * step, l * step};
        const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        double f[3] = {0.0, 0.0, 0.0}, ph = 0.0;
        for (int nx = -3; nx <= 3; nx++)
            for (int ny = -3; ny <= 3; ny++)
                for (int nz = -3; nz <= 3; nz++) {
                    const double sx = d[0] + nx, sy = d[1] + ny, sz = d[2] + nz;
                    const double s2 = sx * sx + sy * sy + sz * sz;
                    const bool centre = nx == 0 && ny == 0 && nz == 0;
                    if (centre && d2 == 0.0) {
                        ph += 2.0 * a / sqpi;  // erf(a s) / s as s -> 0
                        continue;
                    }
                    const double s = sqrt(s2);
                    double g = erfc(a * s) + 2.0 * a * s / sqpi * exp(-a2 * s2);
                    double q = -erfc(a * s) / s;
                    if (centre) {  // the nearest image itself is the walk's
                        g -= 1.0;
                        q += 1.0 / s;
                    }
                    const double w = g / (s2 * s);
                    f[0] += sx * w;
                    f[1] += sy * w;
                    f[2] += sz * w;
                    ph += q;
                }
        for (int mx = -kKmax; mx <= kKmax; mx++)
            for (int my = -kKmax; my <= kKmax; my++)
                for (int mz = -kKmax; mz <= kKmax; mz++) {
                    const double w = c_kweight[((mx + kKmax) * kKw + (my + kKmax)) * kKw + (mz + kKmax)];
                    if (w == 0.0)
                        continue;
                    const double kd = tw * (mx * d[0] + my * d[1] + mz * d[2]);
                    double sn, cs;
                    sincos(kd, &sn, &cs);
                    f[0] += w * tw * mx * sn;
                    f[1] += w * tw * my * sn;
                    f[2] += w * tw * mz * sn;
                    ph -= w * cs;
                }
        ph += kPi / a2;  // pi / (a^2 V) at V = 1
        tab[e] = make_float4((float)f[0], (float)f[1], (float)f[2], (float)ph);
    }
}

}  // namespace

int ewald_table_for(Ctx *c, bool may_alloc, cudaStream_t st, const float4 **tab, float *phi0) {
    {
        std::lock_guard<std::mutex> lk(c->mu);
        if (c->ewald_tab.p) {
            *tab = static_cast<const float4 *>(c->ewald_tab.p);
            *phi0 = c->ewald_phi0;
            return TPM_OK;
        }
    }
    if (!may_alloc) {
        set_error("the Ewald correction table is not built yet: one tpm_compute_forces call on a periodic system "
                  "without treepm builds it");
        return TPM_EINVAL;
    }
    static std::mutex init_mu;
    std::lock_guard<std::mutex> once(init_mu);
    {
        std::lock_guard<std::mutex> lk(c->mu);
        if (c->ewald_tab.p) {
            *tab = static_cast<const float4 *>(c->ewald_tab.p);
            *phi0 = c->ewald_phi0;
            return TPM_OK;
        }
    }
    // k-space weights at unit box: (4 pi / V) e^{-k^2 / 4 a^2} / k^2, a = 2
    double w[kKw * kKw * kKw];
    for (int mx = -kKmax; mx <= kKmax; mx++)
        for (int my = -kKmax; my <= kKmax; my++)
            for (int mz = -kKmax; mz <= kKmax; mz++) {
                const int m2 = mx * mx + my * my + mz * mz;
                const double k2 = 4.0 * kPi * kPi * m2;
                w[((mx + kKmax) * kKw + (my + kKmax)) * kKw + (mz + kKmax)] =
                    (m2 == 0 || m2 > 30) ? 0.0 : 4.0 * kPi * std::exp(-k2 / 16.0) / k2;
            }
    TPM_CUDA(cudaMemcpyToSymbolAsync(c_kweight, w, sizeof w, 0, cudaMemcpyHostToDevice, st));
    const int m = kEwaldN + 1;
    const size_t bytes = (size_t)m * m * m * sizeof(float4);
    void *p = nullptr;
    TPM_CHECK(ctx_alloc(c, &p, bytes, st));
    k_ewald_table<<<(unsigned)(c->num_sms * 4), 128, 0, st>>>(static_cast<float4 *>(p), kEwaldN);
    count_launch();
    float4 first;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&first, p, sizeof first, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        ctx_free(c, p, bytes, st);
        set_error("Ewald table: %s", cudaGetErrorString(e));
        return TPM_ECUDA;
    }
    std::lock_guard<std::mutex> lk(c->mu);
    c->ewald_tab = DevAlloc{p, bytes};
    c->ewald_phi0 = first.w;
    *tab = static_cast<const float4 *>(p);
    *phi0 = first.w;
    return TPM_OK;
}

}  // namespace tpm
