// batched_kernel.cuh -- device code of the persistent batched kernel (the
// force of Eq. 1 with the per-pair arithmetic of Listing 4, Miki & Hanawa,
// Sec. III.A, per system of a ragged batch, optionally driving the whole
// kick-drift-kick leapfrog inside the kernel).  The design is described at
// the top of batched.cu; batched_inst.cu instantiates one (shape, potential)
// pair of the kernel per object file so the shapes compile in parallel, and
// batched.cu holds the planning kernels and the host side.
#pragma once
#include <climits>

#include "nbody_internal.cuh"

namespace nbk {

// Plan words (int64, on the device), written by the planning kernels.
enum PlanWord { kPlanInvalid = 0, kPlanLarge = 1, kPlanLargeItems = 2, kPlanBodies = 3, kPlanWords = 4 };

// Entries of the round-plan table: small systems of up to 32 * kRoundSlots - 1
// bodies (every shape's image capacity is below that).
constexpr int kRoundSlots = 512;

struct BParams {
    int64_t nsys;
    const int64_t* offsets;   // [nsys+1] device
    const float* eps;         // [nsys]
    const int* order;         // [nsys] large systems first, then by size, descending
    const int64_t* plan;      // kPlanWords words
    const int64_t* lprefix;   // [L+1] prefix sums of the large systems' worker counts
    unsigned long long* queue;  // item counter, zeroed before the launch
    unsigned long long* sysbar;  // [nsys] barrier counters of large systems, zeroed before the launch
    unsigned* heartbeat;      // bumped by every CTA as it makes progress
    float* pos;               // [N][3]
    float* vel;               // [N][3] (leapfrog)
    const float* mass;        // [N]
    float* acc;               // [N][3] (force only)
    float* pot;               // [N] or nullptr (force only)
    float dt;
    int64_t steps;            // 0: force only
    int cap;                  // bodies the shared-memory image holds (multiple of 128 when large systems occur)
    int smem;                 // dynamic shared memory of the launch, bytes
    int grid;                 // CTAs of the launch
    int* err;                 // error word
    unsigned short rounds[kRoundSlots];  // round plan of a small system, by its number of 32-body slots
};

// One block of j-pairs [jb, je) against the thread's I i-bodies.  M: zero the
// pair whose j equals the i-body (ib[k] is its index relative to the first
// body of the j-array).  UNI: every body of the system has the mass mu; the
// pair weight then leaves out the multiplication by m_j (11 instead of 12 FP32
// operations per interaction) and the sums are scaled by mu once per body.
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

// The pairs [p0, p1) of a j-array image against the thread's I i-bodies, into
// the FP32 totals t*: FP32 partial sums over blocks of JB pairs (counted from
// p0) folded into t*.  MASK: exclude the self pair; ib[k] is body k's index
// relative to the image (negative or past its end when not in it).  A warp's
// 32 bodies of a slot start at a multiple of 32, ib[k] & ~31, so their 16
// self pairs are known without another register, and only the blocks holding
// them run the masked loop.
template <int I, bool POT, bool MASK, bool UNI, int U, int JB>
__device__ __forceinline__ void image_sum(const float* __restrict__ sj, int p0, int p1, const f2 (&xi)[I],
                                          const f2 (&yi)[I], const f2 (&zi)[I], const int (&ib)[I], f2 eps2,
                                          f2 (&tx)[I], f2 (&ty)[I], f2 (&tz)[I], f2 (&tp)[I]) {
    const ulonglong2* sp = reinterpret_cast<const ulonglong2*>(sj);
    for (int jb = p0; jb < p1; jb += JB) {
        const int je = min(p1, jb + JB);
        f2 ax[I], ay[I], az[I], ap[I];
#pragma unroll
        for (int k = 0; k < I; ++k) ax[k] = ay[k] = az[k] = ap[k] = 0ull;
        bool own = false;
        if (MASK) {
#pragma unroll
            for (int k = 0; k < I; ++k) {
                const int w0 = (ib[k] & ~31) >> 1;  // the warp's first pair (floor, also for negative ib)
                own = own || (w0 < je && w0 + 16 > jb);
            }
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
}

// The two halves (even and odd j) of an accumulator, added.
__device__ __forceinline__ float hsum(f2 v) {
    float a0, a1;
    upk(v, a0, a1);
    return a0 + a1;
}

// Result of body b of a system (g = off + b in the batch) from its sums: the
// acceleration (and potential) of a force-only call, or the kick (and, for a
// small system, the drift) of a leapfrog evaluation.  RES: the system is
// resident, its velocities at sv in shared memory; the drift is applied to the
// image afterwards.  Resident or not, each update is the same FP32 operation.
template <bool POT, bool UNI, bool RES>
__device__ __forceinline__ void finish_body(const BParams& p, float* sv, int b, int64_t g, int64_t ntot, float ax,
                                            float ay, float az, float pt, float mu, float kick, bool drift) {
    if (UNI) {
        ax *= mu;
        ay *= mu;
        az *= mu;
    }
    if (RES) {
        float* v = sv + 3 * b;
        v[0] = fmaf(kick, ax, v[0]);
        v[1] = fmaf(kick, ay, v[1]);
        v[2] = fmaf(kick, az, v[2]);
        return;
    }
    if (!in_range(g, ntot, p.err)) return;
    if (p.steps == 0) {
        p.acc[3 * g + 0] = ax;
        p.acc[3 * g + 1] = ay;
        p.acc[3 * g + 2] = az;
        if (POT) {
            if (UNI) pt *= mu;
            p.pot[g] = -pt;
        }
    } else {
        float vx = p.vel[3 * g + 0], vy = p.vel[3 * g + 1], vz = p.vel[3 * g + 2];
        vx = fmaf(kick, ax, vx);
        vy = fmaf(kick, ay, vy);
        vz = fmaf(kick, az, vz);
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

// Shared memory a small system takes when it stays resident for all steps of
// a leapfrog call: its image and its velocities ([ns][3] floats after the
// image, 16-byte aligned).
__host__ __device__ __forceinline__ int resident_bytes(int ns) {
    return 32 * ((ns + 1) >> 1) + ((12 * ns + 15) & ~15);
}

// The staging area of a shape with T threads and I slots a warp: a split
// round stages at most T * I bodies' partial sums (4 floats each).
__host__ __device__ constexpr int stage_bytes(int T, int I) { return T * I * 16; }

// Where a split task stages its partial sums: component c of body b goes to
// sv[so + c * rb + b], sv being the first float after the image.  rb == 0:
// the task's sums are complete.  (Two integers, as they stay live across the
// pair loop.)
struct Staging {
    int so;  // float offset from sv of the task's segment, less its first staged body
    int rb;  // bodies staged (one component of one segment)
};

// One task of an evaluation of a small system: N slots of 32 bodies (lane l
// takes body b0 + k*stride + l of slot k) against the j-pairs [p0, p1) of the
// system's image.  With st.rb == 0 the sums are complete and the bodies are
// finished here; otherwise they are one segment of their sums and go to the
// staging area for run_small to add up.
template <int T, int N, bool POT, bool MASK, bool UNI, bool RES, int U, int JB>
__device__ __forceinline__ void eval_task(const float* __restrict__ sj, float* sv, int ns, int b0, int stride, int p0,
                                          int p1, f2 eps2, const BParams& p, int64_t off, int64_t ntot, float kick,
                                          bool drift, float mu, const Staging& st) {
    static_assert(T % 32 == 0 && JB % 16 == 0, "a warp's 32 bodies of a slot are 16 consecutive pairs");
    const int lane = threadIdx.x & 31;
    f2 xi[N], yi[N], zi[N];
    int ib[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
        ib[k] = b0 + k * stride + lane;
        const int b = ib[k] < ns ? ib[k] : 0;  // lanes past the end repeat body 0 and write nothing
        const float* s = sj + (b >> 1) * 8 + (b & 1);
        xi[k] = pk(s[0], s[0]);
        yi[k] = pk(s[2], s[2]);
        zi[k] = pk(s[4], s[4]);
    }
    f2 tx[N], ty[N], tz[N], tp[N];
#pragma unroll
    for (int k = 0; k < N; ++k) tx[k] = ty[k] = tz[k] = tp[k] = 0ull;
    image_sum<N, POT, MASK, UNI, U, JB>(sj, p0, p1, xi, yi, zi, ib, eps2, tx, ty, tz, tp);
#pragma unroll
    for (int k = 0; k < N; ++k) {
        if (ib[k] >= ns) continue;
        const float ax = hsum(tx[k]), ay = hsum(ty[k]), az = hsum(tz[k]);
        const float pt = POT ? hsum(tp[k]) : 0.0f;
        if (st.rb != 0) {
            float* d = sv + st.so + ib[k];
            d[0] = ax;
            d[st.rb] = ay;
            d[2 * st.rb] = az;
            if (POT) d[3 * st.rb] = pt;
            continue;
        }
        finish_body<POT, UNI, RES>(p, sv, ib[k], off + ib[k], ntot, ax, ay, az, pt, mu, kick, drift);
    }
}

// eval_task with n (1 to I) slots, the self-pair mask and the equal-mass loop
// chosen at run time.
template <int T, int I, bool POT, bool RES, int U, int JB>
__device__ __forceinline__ void run_task(bool mask, bool uni, int n, const float* __restrict__ sj, float* sv, int ns,
                                         int b0, int stride, int p0, int p1, f2 eps2, const BParams& p, int64_t off,
                                         int64_t ntot, float kick, bool drift, float mu, const Staging& st) {
#define NBK_TASK(N_, M_, U_)                                                                                        \
    eval_task<T, (I >= N_ ? N_ : 1), POT, M_, U_, RES, U, JB>(sj, sv, ns, b0, stride, p0, p1, eps2, p, off, ntot, \
                                                              kick, drift, mu, st)
#define NBK_TASKN(M_, U_)                   \
    if (I >= 4 && n >= 4) {                 \
        NBK_TASK(4, M_, U_);                \
    } else if (I >= 3 && n == 3) {          \
        NBK_TASK(3, M_, U_);                \
    } else if (I >= 2 && n == 2) {          \
        NBK_TASK(2, M_, U_);                \
    } else {                                \
        NBK_TASK(1, M_, U_);                \
    }
    if (mask) {
        if (uni) {
            NBK_TASKN(true, true)
        } else {
            NBK_TASKN(true, false)
        }
    } else {
        if (uni) {
            NBK_TASKN(false, true)
        } else {
            NBK_TASKN(false, false)
        }
    }
#undef NBK_TASKN
#undef NBK_TASK
}

// Position load; CG: through L2 only (ld.global.cg), for positions another
// CTA of this launch wrote (the L1 of this SM may still hold older values).
template <bool CG>
__device__ __forceinline__ float ld_pos(const float* a) {
    return CG ? __ldcg(a) : *a;
}

// Shared-memory image of bodies [g0, g0 + nb) of the batch as j-pairs, an odd
// count padded with a massless body far away.
template <bool CG = false>
__device__ __forceinline__ void load_image(float* sj, const BParams& p, int64_t g0, int nb, int64_t ntot) {
    const int nbp = (nb + 1) & ~1;
    for (int b = threadIdx.x; b < nbp; b += blockDim.x) {
        float x = kPadPos, y = kPadPos, z = kPadPos, m = 0.0f;
        if (b < nb && in_range(g0 + b, ntot, p.err)) {
            const int64_t g = g0 + b;
            x = ld_pos<CG>(p.pos + 3 * g + 0);
            y = ld_pos<CG>(p.pos + 3 * g + 1);
            z = ld_pos<CG>(p.pos + 3 * g + 2);
            m = p.mass[g];
        }
        float* d = sj + (b >> 1) * 8 + (b & 1);
        d[0] = x;
        d[2] = y;
        d[4] = z;
        d[6] = m;
    }
}

// Equal masses throughout the system (the usual ensemble member)?  Every
// thread of the CTA calls this; *mu gets the first body's mass.
__device__ __forceinline__ bool uniform_system(const BParams& p, int64_t off, int ns, int64_t ntot, float* mu) {
    float m0 = 0.0f;
    if (in_range(off, ntot, p.err)) m0 = p.mass[off];
    bool same = true;
    for (int b = threadIdx.x; b < ns; b += blockDim.x)
        if (in_range(off + b, ntot, p.err)) same = same && p.mass[off + b] == m0;
    *mu = m0;
    return __syncthreads_and(same) != 0;
}

// Round plan of a small system of S slots (32-body groups), from the table the
// host builds per shape (BParams::rounds, indexed by S): F full rounds in
// which every warp takes I1 slots against all j-pairs, then the R = S - F*W*I1
// slots left over, either spread (warp w takes slots w, w + W, ... against all
// j-pairs) or split (groups of I2 slots, each group's j-pairs cut into G
// segments, one warp per group and segment, partial sums added up in shared
// memory in segment order).
enum RoundMode { kRoundNone = 0, kRoundSpread = 1, kRoundSplit = 2 };
__host__ __device__ __forceinline__ unsigned short round_entry(int I1, int mode, int I2, int G) {
    return (unsigned short)((I1 - 1) | (mode << 2) | ((I2 - 1) << 4) | ((G - 1) << 6));
}

// A small system, owned by this CTA for all steps of the call.  RES (a
// leapfrog call whose system fits resident_bytes and the staging area):
// positions and velocities are read from global memory once, every kick and
// drift of the call is applied in shared memory, and both are written back
// once at the end, so no evaluation waits on global memory.  Otherwise every
// evaluation kicks (and drifts) the bodies in global memory and reloads the
// image from there.  The two give the same bits.
template <int T, int I, bool POT, int U, int JB, bool RES>
__device__ void run_small(float* sj, const BParams& p, int s, int64_t ntot) {
    constexpr int W = T / 32;
    const int64_t off = p.offsets[s];
    const int ns = (int)(p.offsets[s + 1] - off);
    if (ns <= 0) return;
    const float e = p.eps[s];
    const float eps2s = e * e;
    const f2 eps2 = pk(eps2s, eps2s);
    const int npair = (ns + 1) >> 1;
    float* sv = sj + 8 * npair;                     // RES: the velocities, [ns][3]
    const int so0 = RES ? ((3 * ns + 3) & ~3) : 0;  // the staging area of split tasks, from sv
    const float* stg = sv + so0;
    float mu;
    const bool uni = uniform_system(p, off, ns, ntot, &mu);
    const bool mask = POT || eps2s == 0.0f;  // the self pair must be excluded
    load_image(sj, p, off, ns, ntot);
    if (RES) {
        for (int q = threadIdx.x; q < 3 * ns; q += T) {
            float v = 0.0f;
            if (in_range(off + q / 3, ntot, p.err)) v = p.vel[3 * off + q];
            sv[q] = v;
        }
    }
    const int S = (ns + 31) >> 5;
    const unsigned re = S < kRoundSlots ? p.rounds[S] : round_entry(I, kRoundSpread, 1, 1);
    const int I1 = (int)(re & 3u) + 1, mode = (int)((re >> 2) & 3u), I2 = (int)((re >> 4) & 3u) + 1;
    const int G = (int)((re >> 6) & 15u) + 1;
    const int F = S / (W * I1), R = S - F * W * I1;
    const int sb = F * W * I1 * 32;  // first body of the last round
    const int w = threadIdx.x >> 5;
    const Staging whole = {0, 0};
    __syncthreads();
    for (int64_t ev = 0; ev <= p.steps; ++ev) {
        const float kick = (p.steps == 0) ? 0.0f : ((ev == 0 || ev == p.steps) ? 0.5f * p.dt : p.dt);
        const bool drift = ev < p.steps;
        for (int r = 0; r < F; ++r)
            run_task<T, I, POT, RES, U, JB>(mask, uni, I1, sj, sv, ns, (r * W + w) * I1 * 32, 32, 0, npair, eps2, p,
                                            off, ntot, kick, drift, mu, whole);
        if (mode == kRoundSpread) {
            const int nw = R > w ? (R - w + W - 1) / W : 0;
            if (nw > 0)
                run_task<T, I, POT, RES, U, JB>(mask, uni, nw, sj, sv, ns, sb + 32 * w, T, 0, npair, eps2, p, off,
                                                ntot, kick, drift, mu, whole);
        } else if (mode == kRoundSplit) {
            const int groups = (R + I2 - 1) / I2;
            const int rb = 32 * R;
            if (w < groups * G) {
                const int q = w / G, seg = w - q * G;
                const Staging st = {so0 + seg * (POT ? 4 : 3) * rb - sb, rb};
                run_task<T, I, POT, RES, U, JB>(mask, uni, min(I2, R - q * I2), sj, sv, ns, sb + 32 * q * I2, 32,
                                                seg * npair / G, (seg + 1) * npair / G, eps2, p, off, ntot, kick,
                                                drift, mu, st);
            }
            __syncthreads();  // every segment's partial sums are staged
            constexpr int NC = POT ? 4 : 3;
            for (int rel = threadIdx.x; rel < rb && sb + rel < ns; rel += T) {
                float ax = stg[rel], ay = stg[rb + rel], az = stg[2 * rb + rel];
                float pt = POT ? stg[3 * rb + rel] : 0.0f;
                for (int g = 1; g < G; ++g) {
                    const float* d = stg + g * NC * rb + rel;
                    ax += d[0];
                    ay += d[rb];
                    az += d[2 * rb];
                    if (POT) pt += d[3 * rb];
                }
                const int b = sb + rel;
                if (uni)
                    finish_body<POT, true, RES>(p, sv, b, off + b, ntot, ax, ay, az, pt, mu, kick, drift);
                else
                    finish_body<POT, false, RES>(p, sv, b, off + b, ntot, ax, ay, az, pt, mu, kick, drift);
            }
        }
        __syncthreads();
        if (drift) {
            if (RES) {
                // every thread has read this evaluation's positions: drift the image in place
                for (int b = threadIdx.x; b < ns; b += T) {
                    float* d = sj + (b >> 1) * 8 + (b & 1);
                    d[0] = fmaf(p.dt, sv[3 * b + 0], d[0]);
                    d[2] = fmaf(p.dt, sv[3 * b + 1], d[2]);
                    d[4] = fmaf(p.dt, sv[3 * b + 2], d[4]);
                }
            } else {
                load_image(sj, p, off, ns, ntot);  // the drifted positions of this step
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) atomicAdd(p.heartbeat, 1u);
    }
    if (RES) {
        for (int b = threadIdx.x; b < ns; b += T) {
            if (!in_range(off + b, ntot, p.err)) continue;
            const float* d = sj + (b >> 1) * 8 + (b & 1);
            p.pos[3 * (off + b) + 0] = d[0];
            p.pos[3 * (off + b) + 1] = d[2];
            p.pos[3 * (off + b) + 2] = d[4];
        }
        for (int q = threadIdx.x; q < 3 * ns; q += T)
            if (in_range(off + q / 3, ntot, p.err)) p.vel[3 * off + q] = sv[q];
    }
}

// ---------------------------------------------------------------------------
// Large systems: several CTAs per system, bodies streamed in tiles.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long load_acquire_u64(const unsigned long long* a) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(v) : "l"(a) : "memory");
    return v;
}
__device__ __forceinline__ unsigned load_relaxed_u32(const unsigned* a) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}

// The W workers of one large system meet here once per phase: each CTA adds 1
// to the system's counter and waits until it reaches target = phase * W.  The
// wait is bounded: if the counter is still short while no CTA of the grid has
// bumped the heartbeat for kWaitLimitNs, the wait gives up, records a timeout
// in the error word and returns false (the caller abandons the system).
static __device__ bool system_barrier(const BParams& p, unsigned long long* ctr, unsigned long long target) {
    __shared__ int s_ok;
    __syncthreads();  // every thread's writes of this phase are issued
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1ull);
        int ok = 1;
        unsigned hb = load_relaxed_u32(p.heartbeat);
        uint64_t t0 = globaltimer_ns();
        while (load_acquire_u64(ctr) < target) {
            __nanosleep(256);
            const uint64_t now = globaltimer_ns();
            if (now - t0 > kWaitLimitNs) {
                const unsigned h = load_relaxed_u32(p.heartbeat);
                if (h == hb) {
                    ok = 0;
                    atomicExch(p.err, kErrTimeout);
                    break;
                }
                hb = h;
                t0 = now;
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ void kahan_fold(f2& sum, f2& comp, f2 part) {
    const f2 y = sub2(part, comp);
    const f2 t = add2(sum, y);
    comp = sub2(sub2(t, sum), y);
    sum = t;
}

// One chunk of 2T i-bodies [cb, cb + 2T) of a large system (bodies
// [off, off + ns) of the batch) against all of its bodies, streamed through
// the shared-memory image in tiles of tj bodies (a multiple of 128, so a
// warp's 32 bodies of a slot lie in one tile and one 64-pair block).  Writes
// the acceleration (and potential) or applies the kick; the drift of a large
// system waits for its barrier.
template <int T, bool POT, bool MASK, bool UNI, int U, int JB>
__device__ void large_chunk(float* sj, const BParams& p, int64_t off, int ns, int cb, int tj, f2 eps2, float kick,
                            float mu, int64_t ntot) {
    constexpr int I = 2;
    const int tid = threadIdx.x;
    f2 xi[I], yi[I], zi[I];
    int ib[I];
#pragma unroll
    for (int k = 0; k < I; ++k) {
        ib[k] = cb + k * T + tid;
        const int64_t g = off + (ib[k] < ns ? ib[k] : cb);  // past the end: repeat the chunk's first body
        float x = 0.0f, y = 0.0f, z = 0.0f;
        if (in_range(g, ntot, p.err)) {
            x = ld_pos<true>(p.pos + 3 * g + 0);
            y = ld_pos<true>(p.pos + 3 * g + 1);
            z = ld_pos<true>(p.pos + 3 * g + 2);
        }
        xi[k] = pk(x, x);
        yi[k] = pk(y, y);
        zi[k] = pk(z, z);
    }
    f2 sx[I], sy[I], sz[I], sp[I], cx[I], cy[I], cz[I], cp[I];
#pragma unroll
    for (int k = 0; k < I; ++k) sx[k] = sy[k] = sz[k] = sp[k] = cx[k] = cy[k] = cz[k] = cp[k] = 0ull;
    for (int j0 = 0; j0 < ns; j0 += tj) {
        const int nb = min(tj, ns - j0);
        __syncthreads();  // the previous tile is consumed
        load_image<true>(sj, p, off + j0, nb, ntot);
        __syncthreads();
        int ibr[I];
#pragma unroll
        for (int k = 0; k < I; ++k) ibr[k] = ib[k] - j0;
        f2 tx[I], ty[I], tz[I], tp[I];
#pragma unroll
        for (int k = 0; k < I; ++k) tx[k] = ty[k] = tz[k] = tp[k] = 0ull;
        image_sum<I, POT, MASK, UNI, U, JB>(sj, 0, (nb + 1) >> 1, xi, yi, zi, ibr, eps2, tx, ty, tz, tp);
#pragma unroll
        for (int k = 0; k < I; ++k) {
            kahan_fold(sx[k], cx[k], tx[k]);
            kahan_fold(sy[k], cy[k], ty[k]);
            kahan_fold(sz[k], cz[k], tz[k]);
            if (POT) kahan_fold(sp[k], cp[k], tp[k]);
        }
        if (tid == 0) atomicAdd(p.heartbeat, 1u);
    }
#pragma unroll
    for (int k = 0; k < I; ++k) {
        if (ib[k] >= ns) continue;
        finish_body<POT, UNI, false>(p, nullptr, ib[k], off + ib[k], ntot, hsum(sub2(sx[k], cx[k])),
                                     hsum(sub2(sy[k], cy[k])), hsum(sub2(sz[k], cz[k])), hsum(sub2(sp[k], cp[k])), mu,
                                     kick, false);
    }
}

// Worker w of the W workers of large system s: chunks w, w + W, ... of 2T
// bodies, for every force evaluation of the call.
template <int T, bool POT, int U, int JB>
__device__ void run_large(float* sj, const BParams& p, int s, int w, int W, int64_t ntot) {
    const int64_t off = p.offsets[s];
    const int ns = (int)(p.offsets[s + 1] - off);
    const float e = p.eps[s];
    const float eps2s = e * e;
    const f2 eps2 = pk(eps2s, eps2s);
    float mu;
    const bool uni = uniform_system(p, off, ns, ntot, &mu);
    const int C = 2 * T;
    const int nch = (ns + C - 1) / C;
    const bool mask = POT || eps2s == 0.0f;
    unsigned long long* bar = p.sysbar + s;
    unsigned long long phase = 0;
    for (int64_t ev = 0; ev <= p.steps; ++ev) {
        const float kick = (p.steps == 0) ? 0.0f : ((ev == 0 || ev == p.steps) ? 0.5f * p.dt : p.dt);
        for (int c = w; c < nch; c += W) {
            if (mask) {
                if (uni)
                    large_chunk<T, POT, true, true, U, JB>(sj, p, off, ns, c * C, p.cap, eps2, kick, mu, ntot);
                else
                    large_chunk<T, POT, true, false, U, JB>(sj, p, off, ns, c * C, p.cap, eps2, kick, mu, ntot);
            } else {
                if (uni)
                    large_chunk<T, POT, false, true, U, JB>(sj, p, off, ns, c * C, p.cap, eps2, kick, mu, ntot);
                else
                    large_chunk<T, POT, false, false, U, JB>(sj, p, off, ns, c * C, p.cap, eps2, kick, mu, ntot);
            }
        }
        if (ev < p.steps) {
            // every worker has read the positions of this evaluation ...
            if (!system_barrier(p, bar, ++phase * (unsigned long long)W)) return;
            for (int c = w; c < nch; c += W) {
                const int hi = min(ns, (c + 1) * C);
                for (int b = c * C + (int)threadIdx.x; b < hi; b += T) {
                    const int64_t g = off + b;
                    if (!in_range(g, ntot, p.err)) continue;
                    p.pos[3 * g + 0] = fmaf(p.dt, p.vel[3 * g + 0], p.pos[3 * g + 0]);
                    p.pos[3 * g + 1] = fmaf(p.dt, p.vel[3 * g + 1], p.pos[3 * g + 1]);
                    p.pos[3 * g + 2] = fmaf(p.dt, p.vel[3 * g + 2], p.pos[3 * g + 2]);
                }
            }
            // ... and has drifted its bodies before the next evaluation reads them
            if (!system_barrier(p, bar, ++phase * (unsigned long long)W)) return;
        }
    }
}

// ---------------------------------------------------------------------------
// The persistent kernel.
// ---------------------------------------------------------------------------
template <int T, int I, bool POT, int U, int JB>
__global__ void __launch_bounds__(T, 512 / T) batched_kernel(const BParams p) {
    extern __shared__ __align__(16) float sj[];
    __shared__ unsigned long long s_item;
    if (p.plan[kPlanInvalid] != 0) return;  // a bad batch: nothing is written
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(p.queue, 1ull);
        __syncthreads();
        const unsigned long long k = s_item;
        __syncthreads();
        // The plan words are read again for every item rather than held in
        // registers across the item loop: kept live they pushed the pair loop
        // of the 512-thread shape to a 4-byte spill (128 registers).
        const int64_t L = __ldcg(p.plan + kPlanLarge);
        const int64_t TL = __ldcg(p.plan + kPlanLargeItems);
        const int64_t ntot = __ldcg(p.plan + kPlanBodies);
        if (k >= (unsigned long long)(TL + (p.nsys - L))) break;
        if ((int64_t)k < TL) {
            // large system r of the order, lprefix[r] <= k < lprefix[r + 1]
            int64_t lo = 0, hi = L;
            while (hi - lo > 1) {
                const int64_t mid = (lo + hi) >> 1;
                if (p.lprefix[mid] <= (int64_t)k)
                    lo = mid;
                else
                    hi = mid;
            }
            const int s = p.order[lo];
            if (!in_range(s, p.nsys, p.err)) continue;
            run_large<T, POT, U, JB>(sj, p, s, (int)((int64_t)k - p.lprefix[lo]),
                                     (int)(p.lprefix[lo + 1] - p.lprefix[lo]), ntot);
        } else {
            const int64_t r = L + ((int64_t)k - TL);
            if (!in_range(r, p.nsys, p.err)) continue;
            const int s = p.order[r];
            if (!in_range(s, p.nsys, p.err)) continue;
            const int64_t ns = p.offsets[s + 1] - p.offsets[s];
            if (p.steps > 0 && ns <= p.cap && resident_bytes((int)ns) + stage_bytes(T, I) <= p.smem)
                run_small<T, I, POT, U, JB, true>(sj, p, s, ntot);
            else
                run_small<T, I, POT, U, JB, false>(sj, p, s, ntot);
        }
        __syncthreads();  // the shared image is reused by the next item
    }
}

// The kernel shapes, (threads, i-slots per warp, j-unroll, j-block depth in
// pairs), by shape index (the caller's opts->config).  0: one CTA per SM
// (systems from about 760 bodies up); 2: two CTAs per SM; 1 and 3: smaller
// CTAs; 4 and 5: shape 0 with j-blocks of 32 and 128 pairs (the depth of the
// FP32 partial sums folded into the totals), for the tuner to choose among.
struct BShapeDef {
    int threads, ibodies, unroll, jblock;
};
constexpr int kNumBShapes = 6;
constexpr BShapeDef kBShapes[kNumBShapes] = {{512, 4, 8, 64}, {128, 4, 4, 64}, {256, 4, 4, 64},
                                             {128, 2, 4, 64}, {512, 4, 8, 32}, {512, 4, 8, 128}};

typedef void (*BFn)(const BParams);

// batched_kernel<shape k, potential p>, defined in the object file that
// instantiates it (batched_inst.cu built with NBK_BSHAPE=k, NBK_BPOT=p).
BFn batched_fn_00();
BFn batched_fn_01();
BFn batched_fn_10();
BFn batched_fn_11();
BFn batched_fn_20();
BFn batched_fn_21();
BFn batched_fn_30();
BFn batched_fn_31();
BFn batched_fn_40();
BFn batched_fn_41();
BFn batched_fn_50();
BFn batched_fn_51();
}  // namespace nbk
