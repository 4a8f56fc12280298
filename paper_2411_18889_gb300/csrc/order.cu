// order.cu -- spatial ordering of the bodies for the mixed-precision path.
//
// The force kernel takes each body's coordinates relative to the FP64 centre
// of its cell (a run of `block` consecutive bodies) before the FP32 pair
// arithmetic.  In the caller's order a cell spans the whole system and its
// offsets are as large as the system; ordered along a Morton curve a cell is a
// compact region, its offsets are a cell's size, and the FP32 rounding of the
// offsets -- which dominates the error of close pairs -- shrinks with it.
//
// The order: bodies sorted by the 30-bit Morton index of their position in a
// 1024^3 grid over the FP64 bounding box, ties by body index (a stable LSD
// radix sort of (key, index) with 8-bit digits, so the permutation is
// deterministic).  O(n) work, negligible next to the O(n^2) force.
#include "nbody_internal.cuh"

namespace nbk {
namespace {

constexpr int kBits = 10;       // per axis
constexpr int kRedBlocks = 256;  // bounding-box partials
constexpr int kTileThreads = 256;
constexpr int kTileItems = 8;
constexpr int kTile = kTileThreads * kTileItems;  // elements per radix tile
constexpr int kRadix = 256;

__device__ __forceinline__ unsigned spread3(unsigned v) {  // 10 bits -> every third bit
    unsigned r = 0;
#pragma unroll
    for (int b = 0; b < kBits; ++b) r |= ((v >> b) & 1u) << (3 * b);
    return r;
}

__global__ void __launch_bounds__(256) bbox_partial_kernel(int64_t n, const double* __restrict__ pos,
                                                           double* __restrict__ part) {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int c = 0; c < 3; ++c) {
            const double x = pos[3 * i + c];
            lo[c] = fmin(lo[c], x);
            hi[c] = fmax(hi[c], x);
        }
    __shared__ double s[6][256];
    for (int c = 0; c < 3; ++c) {
        s[c][threadIdx.x] = lo[c];
        s[3 + c][threadIdx.x] = hi[c];
    }
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int c = 0; c < 3; ++c) {
                s[c][threadIdx.x] = fmin(s[c][threadIdx.x], s[c][threadIdx.x + w]);
                s[3 + c][threadIdx.x] = fmax(s[3 + c][threadIdx.x], s[3 + c][threadIdx.x + w]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) part[blockIdx.x * 6 + threadIdx.x] = s[threadIdx.x][0];
}

// Morton key and identity index of each body.
__global__ void __launch_bounds__(256) key_kernel(int64_t n, const double* __restrict__ pos,
                                                  const double* __restrict__ part, unsigned* __restrict__ key,
                                                  int* __restrict__ val) {
    __shared__ double box[6];
    if (threadIdx.x < 6) {
        double v = threadIdx.x < 3 ? 1e300 : -1e300;
        for (int b = 0; b < kRedBlocks; ++b) {
            const double x = part[b * 6 + threadIdx.x];
            v = threadIdx.x < 3 ? fmin(v, x) : fmax(v, x);
        }
        box[threadIdx.x] = v;
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        unsigned k = 0;
        for (int c = 0; c < 3; ++c) {
            const double span = box[3 + c] - box[c];
            int q = span > 0.0 ? (int)((pos[3 * i + c] - box[c]) / span * (1 << kBits)) : 0;
            q = q < 0 ? 0 : (q >= (1 << kBits) ? (1 << kBits) - 1 : q);
            k |= spread3((unsigned)q) << c;
        }
        key[i] = k;
        val[i] = (int)i;
    }
}

// Digit histogram of each tile, stored digit-major: hist[d * ntile + tile].
__global__ void __launch_bounds__(kTileThreads) hist_kernel(int64_t n, const unsigned* __restrict__ key, int shift,
                                                            int ntile, int* __restrict__ hist) {
    __shared__ int h[kRadix];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int k = 0; k < kTileItems; ++k) {
        const int64_t i = base + k * kTileThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(key[i] >> shift) & (kRadix - 1)], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntile + blockIdx.x] = h[threadIdx.x];
}

// In-place exclusive scan of m counts by one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) scan_kernel(int* __restrict__ a, int m) {
    __shared__ int tot[1024];
    const int per = (m + 1023) / 1024;
    const int lo = threadIdx.x * per, hi = min(m, lo + per);
    int s = 0;
    for (int k = lo; k < hi; ++k) s += a[k];
    tot[threadIdx.x] = s;
    __syncthreads();
    for (int w = 1; w < 1024; w <<= 1) {
        const int v = (int)threadIdx.x >= w ? tot[threadIdx.x - w] : 0;
        __syncthreads();
        tot[threadIdx.x] += v;
        __syncthreads();
    }
    int run = tot[threadIdx.x] - s;
    for (int k = lo; k < hi; ++k) {
        const int c = a[k];
        a[k] = run;
        run += c;
    }
}

// Stable scatter of one tile: element ranks among equal digits follow index
// order (warp-level match within a round of 256, warp prefixes across the
// round, running digit offsets across rounds).
__global__ void __launch_bounds__(kTileThreads) scatter_kernel(int64_t n, const unsigned* __restrict__ key_in,
                                                               const int* __restrict__ val_in, int shift, int ntile,
                                                               const int* __restrict__ offs,
                                                               unsigned* __restrict__ key_out,
                                                               int* __restrict__ val_out) {
    constexpr int W = kTileThreads / 32;
    __shared__ int wcount[W][kRadix];
    __shared__ int run[kRadix];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    run[tid] = offs[(int64_t)tid * ntile + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int k = 0; k < kTileItems; ++k) {
        for (int w = 0; w < W; ++w) wcount[w][tid] = 0;
        __syncthreads();
        const int64_t i = base + k * kTileThreads + tid;
        const bool valid = i < n;
        const unsigned kk = valid ? key_in[i] : 0u;
        const int d = valid ? (int)((kk >> shift) & (kRadix - 1)) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wcount[warp][d] = __popc(peers);
        __syncthreads();
        {  // thread tid owns digit tid: warp prefixes, then advance its running offset
            int s = run[tid];
            for (int w = 0; w < W; ++w) {
                const int c = wcount[w][tid];
                wcount[w][tid] = s;
                s += c;
            }
            run[tid] = s;
        }
        __syncthreads();
        if (valid) {
            const int dst = wcount[warp][d] + rank;
            key_out[dst] = kk;
            val_out[dst] = val_in[i];
        }
        __syncthreads();
    }
}

unsigned grid_for(int64_t work) {
    int64_t g = (work + 255) / 256;
    const int64_t cap = (int64_t)current_sms() * 16;
    if (g > cap) g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

size_t order_scratch_bytes(int64_t n) {
    const int64_t ntile = (n + kTile - 1) / kTile;
    return (size_t)n * 16 + (size_t)ntile * kRadix * 4 + kRedBlocks * 6 * 8 + 512;
}

cudaError_t spatial_order(int64_t n, const double* pos, int* perm, void* scratch, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int ntile = (int)((n + kTile - 1) / kTile);
    unsigned char* s = static_cast<unsigned char*>(scratch);
    double* part = reinterpret_cast<double*>(s);
    s += kRedBlocks * 6 * 8;
    unsigned* ka = reinterpret_cast<unsigned*>(s);
    unsigned* kb = ka + n;
    int* va = reinterpret_cast<int*>(kb + n);
    int* vb = va + n;
    int* hist = vb + n;
    bbox_partial_kernel<<<kRedBlocks, 256, 0, st>>>(n, pos, part);
    key_kernel<<<grid_for(n), 256, 0, st>>>(n, pos, part, ka, va);
    for (int pass = 0; pass < 4; ++pass) {  // 30-bit keys, 8 bits per pass
        const int shift = 8 * pass;
        unsigned* kin = (pass & 1) ? kb : ka;
        unsigned* kout = (pass & 1) ? ka : kb;
        int* vin = (pass & 1) ? vb : va;
        int* vout = (pass == 3) ? perm : ((pass & 1) ? va : vb);
        hist_kernel<<<ntile, kTileThreads, 0, st>>>(n, kin, shift, ntile, hist);
        scan_kernel<<<1, 1024, 0, st>>>(hist, ntile * kRadix);
        scatter_kernel<<<ntile, kTileThreads, 0, st>>>(n, kin, vin, shift, ntile, hist, kout, vout);
    }
    return cudaGetLastError();
}

size_t sort_pass_hist_ints(int64_t n) { return (size_t)((n + kTile - 1) / kTile) * kRadix; }

cudaError_t sort_pass(int64_t n, const unsigned* key_in, const int* val_in, int shift, unsigned* key_out,
                      int* val_out, int* hist, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int ntile = (int)((n + kTile - 1) / kTile);
    hist_kernel<<<ntile, kTileThreads, 0, st>>>(n, key_in, shift, ntile, hist);
    scan_kernel<<<1, 1024, 0, st>>>(hist, ntile * kRadix);
    scatter_kernel<<<ntile, kTileThreads, 0, st>>>(n, key_in, val_in, shift, ntile, hist, key_out, val_out);
    return cudaGetLastError();
}

}  // namespace nbk
