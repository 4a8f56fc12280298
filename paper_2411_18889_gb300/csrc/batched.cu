// batched.cu -- many independent systems of uneven size in one persistent
// launch: the force of Eq. 1 (Miki & Hanawa, Sec. III.A, per-pair arithmetic of
// Listing 4) for each system, optionally driving a whole kick-drift-kick
// leapfrog inside the kernel (the integrator is not in the paper).
//
// Planning on the device.  A call queues a few small kernels before the
// persistent one, so it never waits for the host: one validates the offsets
// and softenings (a bad batch sets the error word and nothing is written) and
// gives every system an 8-bit key, large systems first, then the others by
// size in steps of 1/8 octave; one stable radix pass orders the systems by
// that key (longest processing time first, to within 12.5 %); one small
// kernel counts the workers each large system gets.
//
// Scheduling.  A persistent grid of CTAs pulls work items from an atomic
// queue in that order.  A system that fits the CTA's shared-memory image
// ("small") is one item: one CTA owns it for the whole call, and every force
// evaluation and every kick and drift of all steps happen without another
// launch.  A system larger than the image ("large") is W items, W = the
// number of 2*T-body i-chunks it has, at most the grid: its W workers each
// take every W-th chunk and stream the system's bodies through shared
// memory in tiles; between a step's force evaluation and its drift, and
// after the drift, the workers meet at a barrier of their own in global
// memory.  The launch is cooperative whenever a large system can occur, so
// every CTA of the grid is resident and the items of a large system, which
// are contiguous in the queue, are all taken by running CTAs.  The barrier's
// wait is bounded: it gives up (error word, the CTA moves on) only when no
// CTA of the grid has made progress for 4 s, so a long item elsewhere in the
// grid cannot end it early.
//
// Shapes (chosen by the largest system of the batch through the tune table
// when the host knows the sizes; shape 0 otherwise).  From about 760 bodies
// up one 512-thread CTA per SM owns a system (16 warps on one system, up to
// 4 slots of 32 i-bodies a warp); smaller batches run 256- or 128-thread
// CTAs, several per SM, each on its own system.  On GB300 the single large
// CTA ran the ragged 64-to-4096-body workload at 71.7 % of FP32 peak against
// 66.1 % for two 256-thread CTAs per SM.
//
// Rounds.  A system of S slots (32-body groups) runs whole rounds, every warp
// taking I1 slots against all j-pairs, and then its remainder: spread over
// the warps, or, when few slots are left, in groups whose j-pairs are cut
// into segments, one warp per group and segment, the segment sums added in
// shared memory in segment order.  The host picks each S's plan by a cost
// model of the SM's four schedulers fitted on GB300.  A 2112-body system
// no longer runs its last 64 bodies on two warps while 14 wait: on GB300 the
// ragged workload went from 71.1 % to 73.6 % of FP32 peak.
//
// Layout.  Shared memory holds the system (or a tile of a large one) as
// j-pairs (x0,x1,y0,y1,z0,z1,m0,m1): 16 bytes per body, so a 4096-body system
// takes 64 KiB.  In a leapfrog call a small system whose velocities fit
// beside its image (12 more bytes per body) stays resident: every kick and
// drift of the call is applied in shared memory and the state is written back
// once, so no evaluation waits on global memory (on GB300 this lifted
// 256-to-1024-body systems by 3 to 4 points of FP32 peak).  Each thread keeps I i-bodies with their coordinates
// duplicated in f32x2 registers (x_i, x_i); one pair of 16-byte broadcast
// loads gives two j-bodies and each i-body then takes the 12 (13 with the
// potential) packed f32x2 instructions and two MUFU reciprocal square roots
// of Listing 4's sequence, for two interactions.  The two halves of each
// accumulator (even and odd j) are added at the end.
//
// Accumulation.  FP32 partial sums over blocks of 64 j-pairs are folded into
// an FP32 total (two-level summation), so a 4096-term sum carries the rounding
// of two 64-term sums instead of one 4096-term running sum.  Large systems
// add a third level: each tile's FP32 total is folded into the running sum by
// Kahan summation.
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
#include <climits>
#include <cstring>
#include <memory>
#include <mutex>

#include "nbody_internal.cuh"

namespace nbk {
namespace {

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
__device__ bool system_barrier(const BParams& p, unsigned long long* ctr, unsigned long long target) {
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

// ---------------------------------------------------------------------------
// Planning kernels.
// ---------------------------------------------------------------------------
// Sort key of a system: 255 - q, q = 128 + 4 e + (2 bits) for a large system
// of 2^e * 1.xx bodies and q = 8 e + (3 bits) for a small one, so an ascending
// sort puts the large systems first and then every system by size, descending,
// in steps of 1/4 and 1/8 octave.  Empty and one-body systems go last.
__device__ __forceinline__ unsigned size_key(int64_t ns, int cap) {
    if (ns <= 1) return 255u;
    const unsigned n = (unsigned)ns;
    const int e = 31 - __clz(n);
    const unsigned m = e >= 3 ? (n >> (e - 3)) & 7u : (n << (3 - e)) & 7u;
    const unsigned q = ns > cap ? 128u + 4u * (unsigned)e + (m >> 1) : 8u * (unsigned)e + m;
    return 255u - q;
}

// Checks the batch (offsets[0] == 0, sizes >= 0 and below 2^31, softenings
// finite and >= 0), counts the large systems and writes every system's key.
__global__ void __launch_bounds__(256) plan_keys_kernel(int64_t nsys, const int64_t* __restrict__ off,
                                                        const float* __restrict__ eps, int cap,
                                                        unsigned* __restrict__ key, int* __restrict__ val,
                                                        int64_t* __restrict__ plan, int* err) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nsys; s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = off[s], b = off[s + 1];
        const int64_t ns = b - a;
        const float e = eps[s];
        const bool bad = ns < 0 || ns > INT_MAX || !(isfinite(e) && e >= 0.0f) || (s == 0 && a != 0);
        if (bad) {
            atomicExch(reinterpret_cast<unsigned long long*>(plan + kPlanInvalid), 1ull);
            atomicCAS(err, 0, kErrInvalid);
        }
        key[s] = size_key(bad ? 0 : ns, cap);
        val[s] = (int)s;
        if (!bad && ns > cap) atomicAdd(reinterpret_cast<unsigned long long*>(plan + kPlanLarge), 1ull);
        if (s == nsys - 1) plan[kPlanBodies] = b;
    }
}

// Workers of each large system (min(grid, its 2T-body chunks)) and their
// prefix sums over the order; one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) plan_workers_kernel(const int* __restrict__ order,
                                                            const int64_t* __restrict__ off, int64_t* plan,
                                                            int64_t* __restrict__ lprefix, int grid, int chunk) {
    __shared__ int64_t part[1024];
    __shared__ int64_t carry;
    if (plan[kPlanInvalid] != 0) return;
    const int64_t L = plan[kPlanLarge];
    const int tid = threadIdx.x;
    if (tid == 0) {
        carry = 0;
        lprefix[0] = 0;
    }
    __syncthreads();
    for (int64_t base = 0; base < L; base += 1024) {
        const int64_t r = base + tid;
        int64_t wk = 0;
        if (r < L) {
            const int s = order[r];
            const int64_t ns = off[s + 1] - off[s];
            wk = min((int64_t)grid, (ns + chunk - 1) / chunk);
        }
        part[tid] = wk;
        __syncthreads();
        for (int d = 1; d < 1024; d <<= 1) {  // inclusive scan
            const int64_t v = tid >= d ? part[tid - d] : 0;
            __syncthreads();
            part[tid] += v;
            __syncthreads();
        }
        if (r < L) lprefix[r + 1] = carry + part[tid];
        __syncthreads();
        if (tid == 0) carry += part[1023];
        __syncthreads();
    }
    if (tid == 0) plan[kPlanLargeItems] = carry;
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

// Scratch layout (each area 256-byte aligned).
struct BScratch {
    int64_t* plan;               // kPlanWords
    unsigned long long* queue;
    unsigned* heartbeat;
    unsigned* key_a;
    unsigned* key_b;
    int* val_a;
    int* order;
    int* hist;
    int64_t* lprefix;
    unsigned long long* sysbar;
    size_t words_bytes;          // plan + queue + heartbeat, zeroed per call
    size_t total;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

BScratch carve(void* base, int64_t nsys) {
    BScratch b;
    const uintptr_t c = reinterpret_cast<uintptr_t>(base);
    size_t o = 0;
    b.plan = reinterpret_cast<int64_t*>(c + o);
    b.queue = reinterpret_cast<unsigned long long*>(c + o + kPlanWords * 8);
    b.heartbeat = reinterpret_cast<unsigned*>(c + o + kPlanWords * 8 + 8);
    b.words_bytes = kPlanWords * 8 + 16;
    o += align256(b.words_bytes);
    b.key_a = reinterpret_cast<unsigned*>(c + o);
    o += align256((size_t)nsys * 4);
    b.key_b = reinterpret_cast<unsigned*>(c + o);
    o += align256((size_t)nsys * 4);
    b.val_a = reinterpret_cast<int*>(c + o);
    o += align256((size_t)nsys * 4);
    b.order = reinterpret_cast<int*>(c + o);
    o += align256((size_t)nsys * 4);
    b.hist = reinterpret_cast<int*>(c + o);
    o += align256(sort_pass_hist_ints(nsys) * 4);
    b.lprefix = reinterpret_cast<int64_t*>(c + o);
    o += align256((size_t)(nsys + 1) * 8);
    b.sysbar = reinterpret_cast<unsigned long long*>(c + o);
    o += align256((size_t)nsys * 8);
    b.total = o;
    return b;
}

}  // namespace

int batched_num_shapes() { return kNumBShapes; }
BatchShape batched_shape(int k) { return bshapes()[k].shape; }

size_t batched_smem_bytes(int cap) { return (size_t)((cap + 1) / 2) * 8 * sizeof(float); }

size_t batched_scratch_bytes(int64_t nsys) { return carve(nullptr, nsys).total; }

// The shared memory a CTA of shape k may take and still let the CTAs its
// registers allow share an SM; never more than one CTA may hold.
static int cta_smem_limit(int k) {
    const BShapeEntry& e = bshapes()[k];
    int dev = 0, optin = 48 * 1024, per_sm = 48 * 1024, occ = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, e.fn[0], e.shape.threads, 0) != cudaSuccess) {
        (void)cudaGetLastError();
    }
    occ = std::max(occ, 1);
    return std::min(optin, per_sm / occ) - 1024;  // room for static shared memory and the runtime's share
}

int batched_max_cap(int k) {
    const BatchShape sh = bshapes()[k].shape;
    return std::max(128, (cta_smem_limit(k) - stage_bytes(sh.threads, sh.ibodies)) / 16 / 128 * 128);
}

// Round plans.  A cost model of one evaluation of a small system picks, for
// every slot count S, the plan with the least modelled time: a round's time is
// the largest, over the SM's four schedulers (warp w runs on scheduler w % 4),
// of the work its warps hold -- slots times the fraction of j-pairs, each slot
// weighted by kSlotCost[n] for a warp of n slots (fewer i-bodies per thread
// reuse each j-load less) -- divided by kSchedEff[m] for m busy warps (with
// the co-resident CTAs; one warp alone cannot hide its own latency).  A split
// round adds the cost of the staging and its barrier, about 2 us, in units of
// one slot against the whole system.  The constants were fitted to the
// throughput of equal-size batches of 512 to 4096 bodies on GB300 with every
// remainder spread (rms error 1 point of FP32 peak).
static double round_cost(const int* n, const double* f, int ntask, int occ) {
    static const double kSchedEff[5] = {0.0, 0.5, 0.85, 0.95, 1.0};
    static const double kSlotCost[5] = {0.0, 1.1, 1.04, 1.01, 1.0};
    double per[4] = {0.0, 0.0, 0.0, 0.0};
    int cnt[4] = {0, 0, 0, 0};
    for (int w = 0; w < ntask; ++w) {
        if (n[w] <= 0) continue;
        per[w % 4] += n[w] * f[w] * kSlotCost[n[w]];
        cnt[w % 4] += 1;
    }
    double t = 0.0;
    for (int q = 0; q < 4; ++q)
        if (cnt[q] > 0) t = std::max(t, per[q] / kSchedEff[std::min(4, cnt[q] * occ)]);
    return t;
}

static unsigned short plan_rounds(int S, int W, int I, int occ) {
    if (S <= 0) return round_entry(I, kRoundNone, 1, 1);
    const int npair_min = 16 * (S - 1) + 1;  // the smallest system of S slots
    const double comb = 75.0 / npair_min;
    int n[32];
    double f[32];
    double best = 1e300;
    unsigned short entry = round_entry(I, kRoundSpread, 1, 1);
    auto take = [&](double c, unsigned short e) {
        if (c < best - 1e-9) {
            best = c;
            entry = e;
        }
    };
    for (int I1 = I; I1 >= 1; --I1) {
        const int F = S / (W * I1);
        if (F == 0 && I1 < I) break;  // no full round: the same plan as I1 = I
        const int R = S - F * W * I1;
        for (int w = 0; w < W; ++w) {
            n[w] = I1;
            f[w] = 1.0;
        }
        const double full = F * round_cost(n, f, W, occ);
        if (R == 0) {
            take(full, round_entry(I1, kRoundNone, 1, 1));
            continue;
        }
        for (int w = 0; w < W; ++w) {
            n[w] = R > w ? (R - w + W - 1) / W : 0;
            f[w] = 1.0;
        }
        take(full + round_cost(n, f, W, occ), round_entry(I1, kRoundSpread, 1, 1));
        for (int I2 = 1; I2 <= std::min(I, R); ++I2) {
            const int groups = (R + I2 - 1) / I2;
            if (groups > W) continue;
            for (int G = 2; G * groups <= W && G <= 16; ++G) {
                if (npair_min / G < 16) break;
                for (int t = 0; t < groups * G; ++t) {
                    n[t] = std::min(I2, R - (t / G) * I2);
                    f[t] = 1.0 / G;
                }
                take(full + round_cost(n, f, groups * G, occ) + comb, round_entry(I1, kRoundSplit, I2, G));
            }
        }
    }
    return entry;
}

// The table of shape k at occ co-resident CTAs, built once.
static const unsigned short* round_table(int k, int occ) {
    static std::mutex mu;
    static std::unique_ptr<unsigned short[]> tabs[kNumBShapes][5];
    occ = std::min(std::max(occ, 1), 4);
    std::lock_guard<std::mutex> lock(mu);
    std::unique_ptr<unsigned short[]>& t = tabs[k][occ];
    if (!t) {
        const BatchShape sh = bshapes()[k].shape;
        t.reset(new unsigned short[kRoundSlots]);
        for (int S = 0; S < kRoundSlots; ++S) t[S] = plan_rounds(S, sh.threads / 32, sh.ibodies, occ);
    }
    return t.get();
}

cudaError_t batched_launch(int k, const BatchArgs& a, int num_sms, cudaStream_t st, int* launched) {
    *launched = 0;
    const BShapeEntry& e = bshapes()[k];
    const int pot = a.pot != nullptr ? 1 : 0;
    // The image of the largest small system and the staging area; a leapfrog
    // call takes more, up to the CTA's share, so that systems keep their
    // velocities resident too.
    const size_t stage = (size_t)stage_bytes(e.shape.threads, e.shape.ibodies);
    size_t smem = batched_smem_bytes(a.cap) + stage;
    if (a.steps > 0)
        smem = std::max(smem, std::min<size_t>((size_t)resident_bytes(a.cap) + stage, (size_t)cta_smem_limit(k)));
    cudaError_t err = cudaFuncSetAttribute(e.fn[pot], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int occ = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, e.fn[pot], e.shape.threads, smem);
    if (err != cudaSuccess) return err;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    // With large systems possible the grid is the full resident set (the
    // launch is cooperative); otherwise at most one CTA per system.
    const int64_t resident = (int64_t)num_sms * occ;
    const int grid = (int)(a.coop ? resident : std::min<int64_t>(resident, std::max<int64_t>(a.nsys, 1)));
    const BScratch sc = carve(a.scratch, a.nsys);

    err = cudaMemsetAsync(sc.plan, 0, sc.words_bytes, st);
    if (err != cudaSuccess) return err;
    if (a.coop) {
        err = cudaMemsetAsync(sc.sysbar, 0, (size_t)a.nsys * 8, st);
        if (err != cudaSuccess) return err;
    }
    const int64_t kb = std::min<int64_t>((a.nsys + 255) / 256, (int64_t)num_sms * 8);
    plan_keys_kernel<<<(unsigned)std::max<int64_t>(kb, 1), 256, 0, st>>>(a.nsys, a.offsets, a.eps, a.cap, sc.key_a,
                                                                        sc.val_a, sc.plan, a.err);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    *launched += 1;
    err = sort_pass(a.nsys, sc.key_a, sc.val_a, 0, sc.key_b, sc.order, sc.hist, st);
    if (err != cudaSuccess) return err;
    *launched += 3;
    if (a.coop) {
        plan_workers_kernel<<<1, 1024, 0, st>>>(sc.order, a.offsets, sc.plan, sc.lprefix, grid, 2 * e.shape.threads);
        err = cudaGetLastError();
        if (err != cudaSuccess) return err;
        *launched += 1;
    }

    BParams p;
    p.nsys = a.nsys;
    p.offsets = a.offsets;
    p.eps = a.eps;
    p.order = sc.order;
    p.plan = sc.plan;
    p.lprefix = sc.lprefix;
    p.queue = sc.queue;
    p.sysbar = sc.sysbar;
    p.heartbeat = sc.heartbeat;
    p.pos = a.pos;
    p.vel = a.vel;
    p.mass = a.mass;
    p.acc = a.acc;
    p.pot = a.pot;
    p.dt = a.dt;
    p.steps = a.steps;
    p.cap = a.cap;
    p.smem = (int)smem;
    p.grid = grid;
    std::memcpy(p.rounds, round_table(k, occ), sizeof(p.rounds));
    p.err = a.err;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)e.shape.threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = a.coop ? 1 : 0;
    err = cudaLaunchKernelEx(&cfg, e.fn[pot], p);
    if (err != cudaSuccess) return err;
    *launched += 1;
    return cudaSuccess;
}

}  // namespace nbk
