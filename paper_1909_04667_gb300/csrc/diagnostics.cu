// FP64 conservation diagnostics of a force evaluation (paper Sec. 7: the
// momentum and energy checks of a gravity solver): the total force sum_i m_i
// a_i (zero for an exactly symmetric pair interaction; a tree walk leaves a
// residual of the size of its force errors), its scale sum_i m_i |a_i|, the
// potential energy 1/2 sum_i m_i phi_i, and with velocities the kinetic
// energy 1/2 sum_i m_i |v_i|^2 and the momentum sum_i m_i v_i.
//
// Every particle's terms are formed in FP64 with explicit round-to-nearest
// operations; each thread sums a fixed set of particles, each block sums its
// threads in a fixed tree order, and one block sums the blocks' partials in
// block order, so the result is the same bits on every run.
#include <cmath>

#include "tpm_internal.cuh"

namespace tpm {
namespace {

constexpr int kDiagThreads = 256;

__device__ __forceinline__ void block_sum(double (*sh)[kDiagThreads], double (&v)[kDiagSums]) {
    for (int q = 0; q < kDiagSums; q++)
        sh[q][threadIdx.x] = v[q];
    __syncthreads();
    for (int w = kDiagThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < kDiagSums; q++)
                sh[q][threadIdx.x] = __dadd_rn(sh[q][threadIdx.x], sh[q][threadIdx.x + w]);
        __syncthreads();
    }
}

// One partial of each diagnostic sum per block: a fixed grid-stride share of
// the particles, summed per thread in index order and then over the block in
// a fixed tree order, so the result does not depend on scheduling.
__global__ void __launch_bounds__(kDiagThreads)
    k_diag_partial(const float *__restrict__ mass, const float *__restrict__ acc, const float *__restrict__ pot,
                   const double *__restrict__ vel, int64_t n, double *__restrict__ partial) {
    __shared__ double sh[kDiagSums][kDiagThreads];
    double v[kDiagSums] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double m = (double)mass[i];
        const double ax = (double)acc[3 * i], ay = (double)acc[3 * i + 1], az = (double)acc[3 * i + 2];
        v[0] = __dadd_rn(v[0], __dmul_rn(m, ax));
        v[1] = __dadd_rn(v[1], __dmul_rn(m, ay));
        v[2] = __dadd_rn(v[2], __dmul_rn(m, az));
        const double a2 = __dadd_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)), __dmul_rn(az, az));
        v[8] = __dadd_rn(v[8], __dmul_rn(m, __dsqrt_rn(a2)));
        if (pot)
            v[3] = __dadd_rn(v[3], __dmul_rn(0.5 * m, (double)pot[i]));
        if (vel) {
            const double vx = vel[3 * i], vy = vel[3 * i + 1], vz = vel[3 * i + 2];
            const double v2 = __dadd_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)), __dmul_rn(vz, vz));
            v[4] = __dadd_rn(v[4], __dmul_rn(0.5 * m, v2));
            v[5] = __dadd_rn(v[5], __dmul_rn(m, vx));
            v[6] = __dadd_rn(v[6], __dmul_rn(m, vy));
            v[7] = __dadd_rn(v[7], __dmul_rn(m, vz));
        }
    }
    block_sum(sh, v);
    if (threadIdx.x < kDiagSums)
        partial[(size_t)blockIdx.x * kDiagSums + threadIdx.x] = sh[threadIdx.x][0];
}

// One block: thread t sums the partials of blocks t, t + 256, ... in order,
// then the block's tree.
__global__ void __launch_bounds__(kDiagThreads)
    k_diag_final(const double *__restrict__ partial, int nb, double *__restrict__ out) {
    __shared__ double sh[kDiagSums][kDiagThreads];
    double v[kDiagSums] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nb; b += kDiagThreads)
        for (int q = 0; q < kDiagSums; q++)
            v[q] = __dadd_rn(v[q], partial[(size_t)b * kDiagSums + q]);
    block_sum(sh, v);
    if (threadIdx.x < kDiagSums)
        out[threadIdx.x] = sh[threadIdx.x][0];
}

}  // namespace

int diagnostics_device(Ctx *c, const System *s, const float *acc, const float *pot, const double *vel,
                       double *out_host, cudaStream_t st) {
    const int nb = c->num_sms * 2;  // fixed per device: the order of the sums is too
    AllocSet tmp;
    tmp.ctx = c;
    struct Guard {
        AllocSet &t;
        cudaStream_t st;
        ~Guard() { t.release(st); }
    } guard{tmp, st};
    double *partial, *out;
    TPM_CHECK(tmp.get(&partial, (size_t)nb * kDiagSums, st));
    TPM_CHECK(tmp.get(&out, kDiagSums, st));
    k_diag_partial<<<(unsigned)nb, kDiagThreads, 0, st>>>(s->mass, acc, pot, vel, s->n, partial);
    count_launch();
    k_diag_final<<<1, kDiagThreads, 0, st>>>(partial, nb, out);
    count_launch();
    TPM_CUDA(cudaGetLastError());
    TPM_CUDA(cudaMemcpyAsync(out_host, out, kDiagSums * sizeof(double), cudaMemcpyDeviceToHost, st));
    TPM_CUDA(cudaStreamSynchronize(st));
    return TPM_OK;
}

}  // namespace tpm
