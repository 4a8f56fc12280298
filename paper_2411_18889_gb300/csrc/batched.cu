// batched.cu -- many independent systems of uneven size in one persistent
// launch: the force of Eq. 1 (Miki & Hanawa, Sec. III.A, per-pair arithmetic of
// Listing 4) for each system, optionally driving a whole kick-drift-kick
// leapfrog inside the kernel (the integrator is not in the paper).
//
// Scheduling.  A persistent grid of CTAs pulls systems from an atomic queue in
// longest-processing-time-first order (the host sorts by n_s^2), so the few
// large systems start first and the many small ones fill the tail.  One CTA
// owns one system for the whole call: its bodies live in shared memory, and
// every force evaluation and every kick and drift of all steps happen without
// another launch.
//
// Shapes (chosen by the largest system of the batch through the tune table).
// From about 760 bodies up one 512-thread CTA per SM owns a system (16 warps
// on one system, i-passes of 2048 bodies); smaller batches run 256- or
// 128-thread CTAs, several per SM, each on its own system.  On GB300 the
// single large CTA ran the ragged 64-to-4096-body workload at 71.7 % of FP32
// peak against 66.1 % for two 256-thread CTAs per SM.
//
// Layout.  Shared memory holds the system as j-pairs (x0,x1,y0,y1,z0,z1,m0,m1):
// 16 bytes per body, so a 4096-body system takes 64 KiB.  Each thread keeps I
// i-bodies with their coordinates duplicated in f32x2
// registers (x_i, x_i); one pair of 16-byte broadcast loads gives two j-bodies
// and each i-body then takes the 12 (13 with the potential) packed f32x2
// instructions and two MUFU reciprocal square roots of Listing 4's sequence,
// for two interactions.  The two halves of each accumulator (even and odd j)
// are added at the end.
//
// Accumulation.  FP32 partial sums over blocks of 64 j-pairs are folded into
// an FP32 total (two-level summation), so a 4096-term sum carries the rounding
// of two 64-term sums instead of one 4096-term running sum.
//
// Self term.  The pair j = i is excluded exactly, as Eq. 1 states, wherever
// it would change a result: in the potential (it would add m_i/eps, and once
// a partial sum holds that, every later add rounds at its ulp) and for
// eps == 0 (where it is 0 * inf).  A warp's bodies of one pass slot are 32
// consecutive bodies, so their self pairs all fall in one 64-pair block of the
// j-loop; only that block runs the masked loop (the choice is warp-uniform).
// Leapfrog evaluations with eps > 0 need no mask: the difference vector of the
// self pair is exactly zero, so it adds exactly 0 to the acceleration.
#include <algorithm>
#include <mutex>

#include "nbody_internal.cuh"

namespace nbk {
namespace {


struct BParams {
    int64_t nsys;
    const int64_t* offsets;  // [nsys+1] device
    const int* order;        // [nsys] LPT order
    int* queue;              // atomic counter, zeroed before the launch
    float* pos;              // [N][3]
    float* vel;              // [N][3] (leapfrog)
    const float* mass;       // [N]
    const float* eps;        // [nsys]
    float* acc;              // [N][3] (force only)
    float* pot;              // [N] or nullptr (force only)
    float dt;
    int64_t steps;           // 0: force only
    int64_t ntot;            // bodies over all systems
    int* err;                // error word (checked builds record index faults)
};

// One block of j-pairs [jb, je) against the thread's I i-bodies.  M: zero the
// pair whose j equals the i-body (ib[k]).  UNI: every body of the system has
// the mass mu; the pair weight then leaves out the multiplication by m_j (11
// instead of 12 FP32 operations per interaction) and the sums are scaled by
// mu once per body.
template <int I, bool POT, bool M, bool UNI, int U>
__device__ __forceinline__ void jblock(const ulonglong2* __restrict__ sp, int jb, int je, const f2 (&xi)[I],
                                       const f2 (&yi)[I], const f2 (&zi)[I], const int (&ib)[I], f2 eps2,
                                       f2 (&ax)[I], f2 (&ay)[I], f2 (&az)[I], f2 (&ap)[I]) {
#pragma unroll U
    for (int jp = jb; jp < je; ++jp) {
        const ulonglong2 A = sp[2 * jp];
        const ulonglong2 B = sp[2 * jp + 1];
        const f2 xj = A.x, yj = A.y, zj = B.x, mj = B.y;
#pragma unroll
        for (int k = 0; k < I; ++k) {
            const f2 dx = sub2(xj, xi[k]);
            const f2 dy = sub2(yj, yi[k]);
            const f2 dz = sub2(zj, zi[k]);
            f2 r2 = fma2(dx, dx, eps2);
            r2 = fma2(dy, dy, r2);
            r2 = fma2(dz, dz, r2);
            float s0, s1;
            upk(r2, s0, s1);
            float q0 = rsqrt_approx(s0);
            float q1 = rsqrt_approx(s1);
            if (M) {
                if (2 * jp == ib[k]) q0 = 0.0f;
                if (2 * jp + 1 == ib[k]) q1 = 0.0f;
            }
            const f2 ri = pk(q0, q1);
            f2 w = mul2(ri, mul2(ri, ri));
            if (!UNI) w = mul2(w, mj);
            ax[k] = fma2(dx, w, ax[k]);
            ay[k] = fma2(dy, w, ay[k]);
            az[k] = fma2(dz, w, az[k]);
            if (POT) ap[k] = fma2(r2, w, ap[k]);
        }
    }
}

// One pass: I i-bodies per thread (slot k of thread t is body base + k*T + t)
// against every j-pair of the system.  MASK: exclude the self pair, in the
// 64-pair block holding the warp's bodies of each slot.
template <int T, int I, bool POT, bool MASK, bool UNI, int U, int JB>
__device__ __forceinline__ void eval_pass(const float* __restrict__ sj, int npair, int ns, int base, f2 eps2,
                                          const BParams& p, int64_t off, float kick, bool drift, float mu) {
    static_assert(T % 32 == 0 && JB % 16 == 0, "a warp's 32 bodies of a slot lie in one j-block");
    const int tid = threadIdx.x;
    f2 xi[I], yi[I], zi[I];
    int ib[I];
    int selfblk[I];  // first j-pair of the block holding this warp's bodies of slot k
#pragma unroll
    for (int k = 0; k < I; ++k) {
        ib[k] = base + k * T + tid;
        selfblk[k] = (((base + k * T + 32 * (tid >> 5)) >> 1) / JB) * JB;
        const int b = ib[k] < ns ? ib[k] : 0;  // threads past the end repeat body 0 and write nothing
        const float* s = sj + (b >> 1) * 8 + (b & 1);
        xi[k] = pk(s[0], s[0]);
        yi[k] = pk(s[2], s[2]);
        zi[k] = pk(s[4], s[4]);
    }
    f2 tx[I], ty[I], tz[I], tp[I];
#pragma unroll
    for (int k = 0; k < I; ++k) tx[k] = ty[k] = tz[k] = tp[k] = 0ull;
    const ulonglong2* sp = reinterpret_cast<const ulonglong2*>(sj);
    for (int jb = 0; jb < npair; jb += JB) {
        const int je = min(npair, jb + JB);
        f2 ax[I], ay[I], az[I], ap[I];
#pragma unroll
        for (int k = 0; k < I; ++k) ax[k] = ay[k] = az[k] = ap[k] = 0ull;
        bool own = false;
        if (MASK) {
#pragma unroll
            for (int k = 0; k < I; ++k) own = own || selfblk[k] == jb;
        }
        if (own)
            jblock<I, POT, true, UNI, U>(sp, jb, je, xi, yi, zi, ib, eps2, ax, ay, az, ap);
        else
            jblock<I, POT, false, UNI, U>(sp, jb, je, xi, yi, zi, ib, eps2, ax, ay, az, ap);
#pragma unroll
        for (int k = 0; k < I; ++k) {
            tx[k] = add2(tx[k], ax[k]);
            ty[k] = add2(ty[k], ay[k]);
            tz[k] = add2(tz[k], az[k]);
            if (POT) tp[k] = add2(tp[k], ap[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < I; ++k) {
        if (ib[k] >= ns) continue;
        float a0, a1;
        upk(tx[k], a0, a1);
        float ax_ = a0 + a1;
        upk(ty[k], a0, a1);
        float ay_ = a0 + a1;
        upk(tz[k], a0, a1);
        float az_ = a0 + a1;
        if (UNI) {
            ax_ *= mu;
            ay_ *= mu;
            az_ *= mu;
        }
        const int64_t g = off + ib[k];
        if (!in_range(g, p.ntot, p.err)) continue;
        if (p.steps == 0) {
            p.acc[3 * g + 0] = ax_;
            p.acc[3 * g + 1] = ay_;
            p.acc[3 * g + 2] = az_;
            if (POT) {
                upk(tp[k], a0, a1);
                float s = a0 + a1;
                if (UNI) s *= mu;
                p.pot[g] = -s;
            }
        } else {
            float vx = p.vel[3 * g + 0], vy = p.vel[3 * g + 1], vz = p.vel[3 * g + 2];
            vx = fmaf(kick, ax_, vx);
            vy = fmaf(kick, ay_, vy);
            vz = fmaf(kick, az_, vz);
            p.vel[3 * g + 0] = vx;
            p.vel[3 * g + 1] = vy;
            p.vel[3 * g + 2] = vz;
            if (drift) {
                p.pos[3 * g + 0] = fmaf(p.dt, vx, p.pos[3 * g + 0]);
                p.pos[3 * g + 1] = fmaf(p.dt, vy, p.pos[3 * g + 1]);
                p.pos[3 * g + 2] = fmaf(p.dt, vz, p.pos[3 * g + 2]);
            }
        }
    }
}

// eval_pass with I' = min(I, left) i-bodies per thread.
template <int T, int I, bool POT, bool MASK, bool UNI, int U, int JB>
__device__ __forceinline__ void pass_dispatch(int left, const float* __restrict__ sj, int npair, int ns, int base,
                                              f2 eps2, const BParams& p, int64_t off, float kick, bool drift,
                                              float mu) {
    if (I >= 4 && left >= 4) {
        eval_pass<T, (I >= 4 ? 4 : 1), POT, MASK, UNI, U, JB>(sj, npair, ns, base, eps2, p, off, kick, drift, mu);
    } else if (I >= 3 && left >= 3) {
        eval_pass<T, (I >= 3 ? 3 : 1), POT, MASK, UNI, U, JB>(sj, npair, ns, base, eps2, p, off, kick, drift, mu);
    } else if (I >= 2 && left >= 2) {
        eval_pass<T, (I >= 2 ? 2 : 1), POT, MASK, UNI, U, JB>(sj, npair, ns, base, eps2, p, off, kick, drift, mu);
    } else {
        eval_pass<T, 1, POT, MASK, UNI, U, JB>(sj, npair, ns, base, eps2, p, off, kick, drift, mu);
    }
}

// Shared-memory image of system s: j-pairs, an odd count padded with a
// massless body far away.
__device__ __forceinline__ void load_system(float* sj, const BParams& p, int64_t off, int ns) {
    const int nb = (ns + 1) & ~1;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        float x = kPadPos, y = kPadPos, z = kPadPos, m = 0.0f;
        if (b < ns && in_range(off + b, p.ntot, p.err)) {
            const int64_t g = off + b;
            x = p.pos[3 * g + 0];
            y = p.pos[3 * g + 1];
            z = p.pos[3 * g + 2];
            m = p.mass[g];
        }
        float* d = sj + (b >> 1) * 8 + (b & 1);
        d[0] = x;
        d[2] = y;
        d[4] = z;
        d[6] = m;
    }
}

template <int T, int I, bool POT, int U, int JB>
__global__ void __launch_bounds__(T) batched_kernel(const BParams p) {
    extern __shared__ __align__(16) float sj[];
    __shared__ int s_next;
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(p.queue, 1);
        __syncthreads();
        const int k = s_next;
        __syncthreads();
        if (k >= p.nsys) break;
        const int s = p.order[k];
        if (!in_range(s, p.nsys, p.err)) continue;
        const int64_t off = p.offsets[s];
        const int ns = (int)(p.offsets[s + 1] - off);
        if (ns <= 0) continue;
        const float e = p.eps[s];
        const float eps2s = e * e;
        const f2 eps2 = pk(eps2s, eps2s);
        const int npair = (ns + 1) >> 1;
        // Equal masses throughout the system (the usual ensemble member)?
        float mu = 0.0f;
        if (in_range(off, p.ntot, p.err)) mu = p.mass[off];
        bool same = true;
        for (int b = threadIdx.x; b < ns; b += blockDim.x)
            if (in_range(off + b, p.ntot, p.err)) same = same && p.mass[off + b] == mu;
        const bool uni = __syncthreads_and(same) != 0;
        load_system(sj, p, off, ns);
        __syncthreads();
        for (int64_t ev = 0; ev <= p.steps; ++ev) {
            const float kick = (p.steps == 0) ? 0.0f : ((ev == 0 || ev == p.steps) ? 0.5f * p.dt : p.dt);
            const bool drift = ev < p.steps;
            for (int base = 0; base < ns; base += T * I) {
                // Each warp takes only as many i-bodies per thread as it has
                // left in this pass (slot k of lane l is body base + k*T + l),
                // and a warp with none skips the pass: padding costs less than
                // one warp's row of bodies per system, not up to T*I - 1.
                const int lw = ns - base - 32 * (int)(threadIdx.x >> 5);
                const int left = lw <= 0 ? 0 : (lw + T - 1) / T;
                if (left == 0) {
                } else if (POT || eps2s == 0.0f) {  // the self pair must be excluded
                    if (uni)
                        pass_dispatch<T, I, POT, true, true, U, JB>(left, sj, npair, ns, base, eps2, p, off, kick,
                                                                    drift, mu);
                    else
                        pass_dispatch<T, I, POT, true, false, U, JB>(left, sj, npair, ns, base, eps2, p, off, kick,
                                                                     drift, mu);
                } else {
                    if (uni)
                        pass_dispatch<T, I, POT, false, true, U, JB>(left, sj, npair, ns, base, eps2, p, off, kick,
                                                                     drift, mu);
                    else
                        pass_dispatch<T, I, POT, false, false, U, JB>(left, sj, npair, ns, base, eps2, p, off, kick,
                                                                      drift, mu);
                }
            }
            __syncthreads();
            if (drift) {
                load_system(sj, p, off, ns);  // the drifted positions of this step
                __syncthreads();
            }
        }
    }
}

typedef void (*BFn)(const BParams);
struct BShapeEntry {
    BatchShape shape;
    BFn fn[2];  // [pot]
};

template <int T, int I, int U = 4, int JB = 64>
BShapeEntry make_bentry() {
    BShapeEntry e;
    e.shape = BatchShape{T, I};
    e.fn[0] = batched_kernel<T, I, false, U, JB>;
    e.fn[1] = batched_kernel<T, I, true, U, JB>;
    return e;
}

const BShapeEntry* bshapes() {
    static const BShapeEntry table[] = {
        make_bentry<512, 4, 8>(),  // 0: one CTA per SM (large systems)
        make_bentry<128, 4>(),     // 1
        make_bentry<256, 4>(),     // 2: two CTAs per SM (systems below ~1000 bodies)
        make_bentry<128, 2>(),     // 3
    };
    return table;
}
constexpr int kNumBShapes = 4;

}  // namespace

int batched_num_shapes() { return kNumBShapes; }
BatchShape batched_shape(int k) { return bshapes()[k].shape; }

size_t batched_smem_bytes(int max_ns) { return (size_t)((max_ns + 1) / 2) * 8 * sizeof(float); }

cudaError_t batched_launch(int k, const BatchArgs& a, int num_sms, cudaStream_t st) {
    const BShapeEntry& e = bshapes()[k];
    const int pot = a.pot != nullptr ? 1 : 0;
    const size_t smem = std::max<size_t>(batched_smem_bytes(a.max_ns), 16);
    cudaError_t err = cudaFuncSetAttribute(e.fn[pot], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int occ = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, e.fn[pot], e.shape.threads, smem);
    if (err != cudaSuccess) return err;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    BParams p;
    p.nsys = a.nsys;
    p.offsets = a.offsets;
    p.order = a.order;
    p.queue = a.queue;
    p.pos = a.pos;
    p.vel = a.vel;
    p.mass = a.mass;
    p.eps = a.eps;
    p.acc = a.acc;
    p.pot = a.pot;
    p.dt = a.dt;
    p.steps = a.steps;
    p.ntot = a.ntot;
    p.err = a.err;
    const int64_t grid = std::min<int64_t>((int64_t)num_sms * occ, std::max<int64_t>(a.nsys, 1));
    err = cudaMemsetAsync(a.queue, 0, sizeof(int), st);
    if (err != cudaSuccess) return err;
    e.fn[pot]<<<(unsigned)grid, e.shape.threads, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace nbk
