// reduce.cu -- FP64 diagnostics of a state: kinetic energy T = sum m|v|^2/2,
// potential energy W = (1/2) sum m_i phi_i (phi from the force kernel),
// momentum sum m v and net force sum m a (zero by Newton's third law, which
// Eq. 1 of Miki & Hanawa, Sec. III.A, obeys pairwise).
//
// Two deterministic passes: a fixed grid writes per-CTA partial sums, one CTA
// adds them in order.  No atomics, so the result does not depend on timing.
#include "nbody_internal.cuh"

namespace nbk {
namespace {

constexpr int kRedBlocks = 304;
constexpr int kRedThreads = 256;
constexpr int kQ = 8;  // T, W, Px, Py, Pz, Fx, Fy, Fz

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename V>
__global__ void __launch_bounds__(kRedThreads) energy_partial_kernel(int64_t n, const V* __restrict__ vel,
                                                                     const float* __restrict__ mass,
                                                                     const float* __restrict__ acc,
                                                                     const float* __restrict__ pot,
                                                                     double* __restrict__ partial) {
    double q[kQ];
#pragma unroll
    for (int k = 0; k < kQ; ++k) q[k] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double m = mass[i];
        const double vx = vel[3 * i], vy = vel[3 * i + 1], vz = vel[3 * i + 2];
        q[0] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
        q[1] += 0.5 * m * (double)pot[i];
        q[2] += m * vx;
        q[3] += m * vy;
        q[4] += m * vz;
        q[5] += m * (double)acc[3 * i];
        q[6] += m * (double)acc[3 * i + 1];
        q[7] += m * (double)acc[3 * i + 2];
    }
    __shared__ double red[kQ][kRedThreads / 32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < kQ; ++k) {
        const double s = warp_sum(q[k]);
        if (l == 0) red[k][w] = s;
    }
    __syncthreads();
    if (threadIdx.x < kQ) {
        double s = 0.0;
        for (int k = 0; k < kRedThreads / 32; ++k) s += red[threadIdx.x][k];
        partial[(int64_t)blockIdx.x * kQ + threadIdx.x] = s;
    }
}

__global__ void energy_final_kernel(const double* __restrict__ partial, int nblocks, double* __restrict__ out9) {
    if (threadIdx.x < kQ) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partial[b * kQ + threadIdx.x];
        // out9 layout: T, W, E, Px, Py, Pz, Fx, Fy, Fz
        const int dst = threadIdx.x < 2 ? threadIdx.x : threadIdx.x + 1;
        out9[dst] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) out9[2] = out9[0] + out9[1];
}

template <typename V>
cudaError_t energy_reduce(int64_t n, const V* vel, const float* mass, const float* acc, const float* pot,
                          double* scratch, double* out9, cudaStream_t st) {
    energy_partial_kernel<V><<<kRedBlocks, kRedThreads, 0, st>>>(n, vel, mass, acc, pot, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    energy_final_kernel<<<1, 32, 0, st>>>(scratch, kRedBlocks, out9);
    return cudaGetLastError();
}

}  // namespace

size_t reduce_scratch_doubles() { return (size_t)kRedBlocks * kQ; }

cudaError_t energy_reduce_f64(int64_t n, const double* vel, const float* mass, const float* acc, const float* pot,
                              double* scratch, double* out9, cudaStream_t st) {
    return energy_reduce<double>(n, vel, mass, acc, pot, scratch, out9, st);
}

cudaError_t energy_reduce_f32(int64_t n, const float* vel, const float* mass, const float* acc, const float* pot,
                              double* scratch, double* out9, cudaStream_t st) {
    return energy_reduce<float>(n, vel, mass, acc, pot, scratch, out9, st);
}

}  // namespace nbk
