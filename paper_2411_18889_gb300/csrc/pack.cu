// pack.cu -- O(n) kernels around the force evaluation: the leapfrog's kick
// and drift (the integrator is not in the paper; the force it drives is
// Eq. 1 of Miki & Hanawa, Sec. III.A) fused with the build of the packed
// j-array the force kernel streams.
//
// Mixed precision: positions and velocities stay FP64; each cell of `block`
// bodies gets an FP64 centre (the mean of its bodies' positions) and the
// packed array holds FP32 offsets from that centre, so the FP32 pair math
// never sees a large absolute coordinate.  Plain precision: FP32 absolute
// coordinates.
#include "nbody_internal.cuh"

namespace nbk {
namespace {

__device__ __forceinline__ void store_jdup(float* jdup, int64_t k, float x, float y, float z, float m) {
    float4* d = reinterpret_cast<float4*>(jdup + k * kJdupFloats);
    d[0] = make_float4(x, x, y, y);
    d[1] = make_float4(z, z, m, m);
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The FP64 pack runs as two body-parallel kernels (one thread per slot of the
// packed array, 256-slot chunks), so at mid sizes it is not bound by a few
// CTAs walking whole cells (one CTA per cell took 23 to 61 us at N = 16384
// against 2 to 3 us now):
//  1. kick (vel += kick * acc, the acceleration from acc or from the force
//     launch's deferred partial sums), drift (pos += drift * vel), and each
//     chunk's FP64 position sum; plain precision writes the packed entry here;
//  2. (mixed) each cell's FP64 centre, the mean of its bodies' positions from
//     its chunk sums in chunk order, and the packed FP32 offsets from it.
// kick/drift == 0 or vel/acc == nullptr skip them; mass == nullptr packs zero
// masses (sinks that exert nothing).  The chunk sums live after the cell
// centres (pack_centre_doubles).
constexpr int kChunk = 256;

template <int NB>
__global__ void __launch_bounds__(kChunk, NB > 8 ? 1 : 2) pack_step_kernel(int64_t n, double* __restrict__ pos,
                                                           double* __restrict__ vel, const float* __restrict__ acc,
                                                           const float* __restrict__ mass, double kick, double drift,
                                                           int plain, float* __restrict__ jdup,
                                                           double* __restrict__ chunks, const int* __restrict__ perm,
                                                           int* __restrict__ err, const SplitSums ss) {
    pdl_trigger();
    pdl_wait();  // the force kernel's accelerations (or partial sums) are complete
    __shared__ double red[3][kChunk / 32];
    const int tid = threadIdx.x;
    const int64_t k = (int64_t)blockIdx.x * kChunk + tid;
    const BlockSplit bs = block_split(ss, (int64_t)blockIdx.x * kChunk);
    double x = 0.0, y = 0.0, z = 0.0;
    if (k < n) {
        int64_t g = perm != nullptr ? perm[k] : k;  // body in slot k
        if (!in_range(g, n, err)) g = k;
        x = ld_chain(pos + 3 * g + 0);
        y = ld_chain(pos + 3 * g + 1);
        z = ld_chain(pos + 3 * g + 2);
        if (vel != nullptr && (kick != 0.0 || drift != 0.0)) {
            double vx = ld_chain(vel + 3 * g + 0), vy = ld_chain(vel + 3 * g + 1), vz = ld_chain(vel + 3 * g + 2);
            if (acc != nullptr && kick != 0.0) {
                float a3[3];
                split_acc<NB>(ss, bs, k, g, acc, a3);
                vx += kick * (double)a3[0];
                vy += kick * (double)a3[1];
                vz += kick * (double)a3[2];
                vel[3 * g + 0] = vx;
                vel[3 * g + 1] = vy;
                vel[3 * g + 2] = vz;
            }
            if (drift != 0.0) {
                x += drift * vx;
                y += drift * vy;
                z += drift * vz;
                pos[3 * g + 0] = x;
                pos[3 * g + 1] = y;
                pos[3 * g + 2] = z;
            }
        }
        if (plain) store_jdup(jdup, k, (float)x, (float)y, (float)z, mass != nullptr ? mass[g] : 0.0f);
    } else if (plain) {
        store_jdup(jdup, k, kPadPos, kPadPos, kPadPos, 0.0f);
    }
    if (plain) return;
    x = warp_sum(x);
    y = warp_sum(y);
    z = warp_sum(z);
    const int w = tid >> 5, l = tid & 31;
    if (l == 0) {
        red[0][w] = x;
        red[1][w] = y;
        red[2][w] = z;
    }
    __syncthreads();
    if (tid < 3) {
        double t = 0.0;
        for (int q = 0; q < kChunk / 32; ++q) t += red[tid][q];
        chunks[3 * (int64_t)blockIdx.x + tid] = t;
    }
}

__global__ void __launch_bounds__(kChunk) pack_offsets_kernel(int64_t n, int block, const double* __restrict__ pos,
                                                              const float* __restrict__ mass,
                                                              float* __restrict__ jdup, double* __restrict__ centres,
                                                              const double* __restrict__ chunks,
                                                              const int* __restrict__ perm, int* __restrict__ err) {
    pdl_trigger();
    pdl_wait();  // every chunk's positions and sums are written
    __shared__ double cen[3];
    const int tid = threadIdx.x;
    const int64_t ch = blockIdx.x;
    const int per_cell = block / kChunk;
    const int64_t cell = ch / per_cell;
    if (tid < 3) {
        double t = 0.0;
        for (int q = 0; q < per_cell; ++q) t += ld_chain(chunks + 3 * (cell * per_cell + q) + tid);
        const int64_t base = cell * block;
        const int64_t cnt = (n - base) < block ? (n - base) : (int64_t)block;
        cen[tid] = t / (double)cnt;
        if (ch % per_cell == 0) centres[3 * cell + tid] = cen[tid];
    }
    __syncthreads();
    const int64_t k = ch * kChunk + tid;
    if (k < n) {
        int64_t g = perm != nullptr ? perm[k] : k;
        if (!in_range(g, n, err)) g = k;
        store_jdup(jdup, k, (float)(ld_chain(pos + 3 * g + 0) - cen[0]), (float)(ld_chain(pos + 3 * g + 1) - cen[1]),
                   (float)(ld_chain(pos + 3 * g + 2) - cen[2]), mass != nullptr ? mass[g] : 0.0f);
    } else {
        store_jdup(jdup, k, kPadPos, kPadPos, kPadPos, 0.0f);
    }
}

// Mixed precision, every pack of a leapfrog call after its first: one kernel
// instead of two.  The centre of a cell is the mean of its bodies' positions
// one step earlier, from the chunk sums the previous pack left in chunks_in
// (a call keeps its bodies in the same cells), so the packed offsets are
// written in the same pass as the kick and the drift; the new positions' chunk
// sums go to chunks_out for the next pack.  Any FP64 point near a cell serves
// as its centre: the lag moves it by one drift, |v| dt, well inside the cell.
// The centre is computed exactly as pack_offsets_kernel computes it (the same
// sums in the same order).
//
// The kernel sits between two force launches on the critical path of a step,
// so it is arranged for latency: the work that needs nothing the previous
// kernels of the call write -- the split of the block's partial sums
// (arithmetic on the launch parameters), the Morton permutation and the
// masses (fixed for the call, written before its first kernel) -- is done
// before the dependency wait; after it, the chunk sums, the state and the
// partial sums are all requested before any of them is used.
constexpr int kMaxChunksPerCell = 8;  // blocks of up to 2048 bodies

template <int NB>
__global__ void __launch_bounds__(kChunk, NB > 8 ? 1 : 2) pack_lagged_kernel(int64_t n, int block, double* __restrict__ pos,
                                                             double* __restrict__ vel, const float* __restrict__ acc,
                                                             const float* __restrict__ mass, double kick,
                                                             double drift, float* __restrict__ jdup,
                                                             double* __restrict__ centres,
                                                             const double* __restrict__ chunks_in,
                                                             double* __restrict__ chunks_out,
                                                             const int* __restrict__ perm, int* __restrict__ err,
                                                             const SplitSums ss) {
    pdl_trigger();
    __shared__ double cin[3 * kMaxChunksPerCell];
    __shared__ double cen[3];
    __shared__ float redf[3][kChunk / 32];
    const int tid = threadIdx.x;
    const int64_t ch = blockIdx.x;
    const int per_cell = block / kChunk;
    const int64_t cell = ch / per_cell;
    const int64_t k = ch * kChunk + tid;
    const BlockSplit bs = block_split(ss, ch * kChunk);
    int64_t g = k;
    float m = 0.0f;
    if (k < n) {
        g = perm != nullptr ? perm[k] : k;  // body in slot k
        if (!in_range(g, n, err)) g = k;
        m = mass != nullptr ? mass[g] : 0.0f;
    }
    pdl_wait();  // the force kernel's results and the previous pack's chunk sums are complete
    if (tid < 3 * per_cell) cin[tid] = ld_chain(chunks_in + 3 * cell * per_cell + tid);
    double x = 0.0, y = 0.0, z = 0.0;
    if (k < n) {
        double vx = ld_chain(vel + 3 * g + 0), vy = ld_chain(vel + 3 * g + 1), vz = ld_chain(vel + 3 * g + 2);
        x = ld_chain(pos + 3 * g + 0);
        y = ld_chain(pos + 3 * g + 1);
        z = ld_chain(pos + 3 * g + 2);
        float a3[3];
        split_acc<NB>(ss, bs, k, g, acc, a3);
        vx += kick * (double)a3[0];
        vy += kick * (double)a3[1];
        vz += kick * (double)a3[2];
        vel[3 * g + 0] = vx;
        vel[3 * g + 1] = vy;
        vel[3 * g + 2] = vz;
        x += drift * vx;
        y += drift * vy;
        z += drift * vz;
        pos[3 * g + 0] = x;
        pos[3 * g + 1] = y;
        pos[3 * g + 2] = z;
    }
    __syncthreads();  // the cell's chunk sums are in shared memory
    if (tid < 3) {
        double t = 0.0;
        for (int q = 0; q < per_cell; ++q) t += cin[3 * q + tid];
        const int64_t base = cell * block;
        const int64_t cnt = (n - base) < block ? (n - base) : (int64_t)block;
        cen[tid] = t / (double)cnt;
        if (ch % per_cell == 0) centres[3 * cell + tid] = cen[tid];
    }
    __syncthreads();
    float ox = 0.0f, oy = 0.0f, oz = 0.0f;
    if (k < n) {
        ox = (float)(x - cen[0]);
        oy = (float)(y - cen[1]);
        oz = (float)(z - cen[2]);
        store_jdup(jdup, k, ox, oy, oz, m);
    } else {
        store_jdup(jdup, k, kPadPos, kPadPos, kPadPos, 0.0f);
    }
    // The chunk's position sum for the next step's centres: its body count
    // times this centre plus the FP32 sum of its offsets.  Any point near the
    // cell serves as a centre, so the offsets' rounding does not matter, and
    // the FP64 pipe (1/64 of the FP32 rate) is left out of the reduction.
    ox = warp_sum_f(ox);
    oy = warp_sum_f(oy);
    oz = warp_sum_f(oz);
    const int w = tid >> 5, l = tid & 31;
    if (l == 0) {
        redf[0][w] = ox;
        redf[1][w] = oy;
        redf[2][w] = oz;
    }
    __syncthreads();
    if (tid < 3) {
        float t = 0.0f;
        for (int q = 0; q < kChunk / 32; ++q) t += redf[tid][q];
        const int64_t left = n - ch * kChunk;
        const int64_t cnt = left < 0 ? 0 : (left < kChunk ? left : (int64_t)kChunk);
        chunks_out[3 * ch + tid] = (double)cnt * cen[tid] + (double)t;
    }
}

// FP32 state, absolute coordinates: one thread per slot (256-slot chunks).
__global__ void __launch_bounds__(kChunk, 2) pack_f32_kernel(int64_t n, float* __restrict__ pos,
                                                          float* __restrict__ vel, const float* __restrict__ acc,
                                                          const float* __restrict__ mass, float kick, float drift,
                                                          float* __restrict__ jdup, const SplitSums ss) {
    pdl_trigger();
    pdl_wait();  // the force kernel's accelerations (or partial sums) are complete
    const int64_t g = (int64_t)blockIdx.x * kChunk + threadIdx.x;
    const BlockSplit bs = block_split(ss, (int64_t)blockIdx.x * kChunk);
    if (g < n) {
        float x = ld_chain(pos + 3 * g + 0), y = ld_chain(pos + 3 * g + 1), z = ld_chain(pos + 3 * g + 2);
        if (vel != nullptr && (kick != 0.0f || drift != 0.0f)) {
            float vx = ld_chain(vel + 3 * g + 0), vy = ld_chain(vel + 3 * g + 1), vz = ld_chain(vel + 3 * g + 2);
            if (acc != nullptr && kick != 0.0f) {
                float a3[3];
                split_acc<16>(ss, bs, g, g, acc, a3);
                vx = fmaf(kick, a3[0], vx);
                vy = fmaf(kick, a3[1], vy);
                vz = fmaf(kick, a3[2], vz);
                vel[3 * g + 0] = vx;
                vel[3 * g + 1] = vy;
                vel[3 * g + 2] = vz;
            }
            if (drift != 0.0f) {
                x = fmaf(drift, vx, x);
                y = fmaf(drift, vy, y);
                z = fmaf(drift, vz, z);
                pos[3 * g + 0] = x;
                pos[3 * g + 1] = y;
                pos[3 * g + 2] = z;
            }
        }
        store_jdup(jdup, g, x, y, z, mass != nullptr ? mass[g] : 0.0f);
    } else {
        store_jdup(jdup, g, kPadPos, kPadPos, kPadPos, 0.0f);
    }
}

// Clears *flag if any mass differs from mass[0]; the flag starts at nonzero.
__global__ void uniform_mass_kernel(int64_t n, const float* __restrict__ mass, int* __restrict__ flag) {
    const float m0 = mass[0];
    bool same = true;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
        same = same && mass[g] == m0;
    if (__syncthreads_or(!same) && threadIdx.x == 0) *flag = 0;
}

template <typename V>
__global__ void kick_kernel(int64_t n3, V* __restrict__ vel, const float* __restrict__ acc, V kick) {
    pdl_trigger();
    pdl_wait();  // the accelerations are complete
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n3; k += (int64_t)gridDim.x * blockDim.x)
        vel[k] += kick * (V)ld_chain(acc + k);
}

}  // namespace

// Threads of a one-CTA-per-cell pack kernel: a thread per body up to 1024, so
// a few large cells still keep many loads in flight.
int pack_threads(int block) { return block >= 1024 ? 1024 : (block < 32 ? 32 : block); }

namespace {

unsigned grid_for(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)current_sms() * 32;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

}  // namespace

// The pack kernels come in two variants that give the same bits: with 16
// partial-sum loads in flight per body (one round of L2 latency for the ~20
// CTAs' partials of a mid-size block; about 180 registers, one CTA per SM)
// when the launch has at most one CTA per SM anyway, and with 8 (two CTAs per
// SM, to hide the latency of the state gathers) when it has more.  At
// N = 2^20 (4096 CTAs) a pack took 143 us with the one-CTA variant and 99 us
// with the two-CTA one (CUDA events, GB300).
static bool few_chunks(unsigned nch) { return nch <= (unsigned)current_sms(); }

size_t pack_centre_doubles(int64_t npad, int block) { return 3 * (size_t)(npad / block) + 3 * (size_t)(npad / kChunk); }

size_t pack_chunk_doubles(int64_t npad) { return 3 * (size_t)(npad / kChunk); }

int pack_f64_launches(bool plain) { return plain ? 1 : 2; }

cudaError_t pack_f64(int64_t n, int64_t npad, int block, double* pos, double* vel, const float* acc,
                     const float* mass, double kick, double drift, bool plain, float* jdup, double* centres,
                     cudaStream_t st, const int* perm, int* err, const SplitSums* ss) {
    if (block % kChunk != 0 || npad % block != 0) return cudaErrorInvalidValue;
    const unsigned nch = (unsigned)(npad / kChunk);
    double* chunks = centres + 3 * (npad / block);
    cudaError_t e = launch_pdl(few_chunks(nch) ? pack_step_kernel<16> : pack_step_kernel<8>, dim3(nch), dim3(kChunk), 0,
                               st, n, pos, vel, acc, mass, kick, drift, plain ? 1 : 0, jdup, chunks, perm, err,
                               ss != nullptr ? *ss : SplitSums());
    if (e != cudaSuccess || plain) return e;
    return launch_pdl(pack_offsets_kernel, dim3(nch), dim3(kChunk), 0, st, n, block, (const double*)pos, mass, jdup,
                      centres, (const double*)chunks, perm, err);
}

cudaError_t pack_f64_lagged(int64_t n, int64_t npad, int block, double* pos, double* vel, const float* acc,
                            const float* mass, double kick, double drift, float* jdup, double* centres,
                            const double* chunks_in, double* chunks_out, cudaStream_t st, const int* perm, int* err,
                            const SplitSums* ss) {
    if (block % kChunk != 0 || block / kChunk > kMaxChunksPerCell || npad % block != 0 || vel == nullptr ||
        acc == nullptr)
        return cudaErrorInvalidValue;
    const unsigned nch = (unsigned)(npad / kChunk);
    return launch_pdl(few_chunks(nch) ? pack_lagged_kernel<16> : pack_lagged_kernel<8>, dim3(nch), dim3(kChunk), 0,
                      st, n, block, pos, vel, acc, mass, kick, drift, jdup, centres, chunks_in, chunks_out, perm, err,
                      ss != nullptr ? *ss : SplitSums());
}

cudaError_t pack_f32(int64_t n, int64_t npad, float* pos, float* vel, const float* acc, const float* mass,
                     float kick, float drift, float* jdup, cudaStream_t st, const SplitSums* ss) {
    if (npad % kChunk != 0) return cudaErrorInvalidValue;
    return launch_pdl(pack_f32_kernel, dim3((unsigned)(npad / kChunk)), dim3(kChunk), 0, st, n, pos, vel, acc, mass,
                      kick, drift, jdup, ss != nullptr ? *ss : SplitSums());
}

cudaError_t uniform_mass_flag(int64_t n, const float* mass, int* flag, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(flag, 1, sizeof(int), st);
    if (e != cudaSuccess) return e;
    const unsigned cap = (unsigned)current_sms() * 4u;
    const unsigned g = grid_for(n, 256);
    uniform_mass_kernel<<<g < cap ? g : cap, 256, 0, st>>>(n, mass, flag);
    return cudaGetLastError();
}

cudaError_t kick_f64(int64_t n, double* vel, const float* acc, double kick, cudaStream_t st) {
    return launch_pdl(kick_kernel<double>, dim3(grid_for(3 * n, 256)), dim3(256), 0, st, 3 * n, vel, acc, kick);
}

cudaError_t kick_f32(int64_t n, float* vel, const float* acc, float kick, cudaStream_t st) {
    return launch_pdl(kick_kernel<float>, dim3(grid_for(3 * n, 256)), dim3(256), 0, st, 3 * n, vel, acc, kick);
}

}  // namespace nbk
