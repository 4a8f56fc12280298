// nbody_internal.cuh -- device helpers and launch interfaces shared by the
// library's translation units (not installed, not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "../../include/nbody.h"

namespace nbk {

// ---------------------------------------------------------------------------
// Layout of the packed j-array ("jdup"), written by the pack kernels and read
// by the force kernel through shared memory:
//   jdup[k] = (x, x, y, y, z, z, m, m)  (8 floats = 32 bytes per body)
// Each coordinate appears twice so that one 64-bit shared load yields the
// broadcast operand of a packed f32x2 instruction acting on two i-bodies.
// Coordinates are relative to the FP64 centre of the body's cell (mixed
// precision) or absolute (plain).  Padding bodies beyond n sit at kPadPos with
// zero mass: their contribution underflows to exactly zero.
// ---------------------------------------------------------------------------
constexpr float kPadPos = 1.0e15f;
constexpr int kJdupFloats = 8;

// Work split of the all-pairs kernels: the (i-block, j) plane is cut into
// granules of kGranule consecutive j-bodies of one i-block row, and CTA c of
// a persistent grid of P takes granules [c*U/P, (c+1)*U/P) of the U in all
// (i-block-major): every CTA gets the same number of pair interactions to
// within one granule, whatever n and P are.  j-tiles are whole multiples of
// a granule, so a CTA's first and last tiles may be used in part.
constexpr int kGranule = 32;

// ---------------------------------------------------------------------------
// Packed FP32 pairs (PTX f32x2 arithmetic, sm_100 and later).  A pair is a
// 64-bit register holding (lo, hi); every op is round-to-nearest with
// flush-to-zero, the fast-math setting the paper's N-body runs use.
// ---------------------------------------------------------------------------
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

#ifndef NBODY_SCALAR_PAIRS
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 r;
    asm("add.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 r;
    asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
#else
// The same operations as two scalar instructions each (for comparison runs).
#define NBK_SCALAR2(name, op)                                                  \
    __device__ __forceinline__ f2 name(f2 a, f2 b) {                           \
        float a0, a1, b0, b1, r0, r1;                                          \
        upk(a, a0, a1);                                                        \
        upk(b, b0, b1);                                                        \
        asm(op ".rn.ftz.f32 %0, %1, %2;" : "=f"(r0) : "f"(a0), "f"(b0));       \
        asm(op ".rn.ftz.f32 %0, %1, %2;" : "=f"(r1) : "f"(a1), "f"(b1));       \
        return pk(r0, r1);                                                     \
    }
NBK_SCALAR2(add2, "add")
NBK_SCALAR2(sub2, "sub")
NBK_SCALAR2(mul2, "mul")
#undef NBK_SCALAR2
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    float a0, a1, b0, b1, c0, c1, r0, r1;
    upk(a, a0, a1);
    upk(b, b0, b1);
    upk(c, c0, c1);
    asm("fma.rn.ftz.f32 %0, %1, %2, %3;" : "=f"(r0) : "f"(a0), "f"(b0), "f"(c0));
    asm("fma.rn.ftz.f32 %0, %1, %2, %3;" : "=f"(r1) : "f"(a1), "f"(b1), "f"(c1));
    return pk(r0, r1);
}
#endif

// Hardware approximate reciprocal square root (MUFU), flush-to-zero.
__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ---------------------------------------------------------------------------
// mbarrier + 1-D bulk copy (TMA) helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Global copy of `bytes` (multiple of 16, both addresses 16-byte aligned) into
// shared memory, completing on `bar` by transaction count.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Every device-side wait gives up after this long, sets the error word and
// lets the kernel return (no trap, no endless spin).
constexpr uint64_t kWaitLimitNs = 4000000000ull;
constexpr int kErrTimeout = 1;
constexpr int kErrBounds = 2;
constexpr int kErrInvalid = 3;  // a batch's offsets or softenings, checked on the device

// Checked builds (-DNBODY_CHECKS, the stand-in for a memory sanitizer): every
// computed global index is tested before use; an index out of range records
// kErrBounds in the error word and the access is skipped.  In normal builds
// the test folds away.
#ifdef NBODY_CHECKS
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif
__device__ __forceinline__ bool in_range(int64_t i, int64_t n, int* err) {
    if (!kChecked) return true;
    if (i >= 0 && i < n) return true;
    if (err != nullptr) atomicCAS(err, 0, kErrBounds);
    return false;
}

// Wait for phase `parity` of `bar`; false if the limit expired.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0 && globaltimer_ns() - t0 > limit_ns) return false;
    }
}

// An NVTX range around each public call, so that a timeline tool shows the
// library's calls by name around their kernels (a no-op without a tool).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define NB_RANGE(name) ::nbk::NvtxRange nb_range_(name)

// SM count of the current device (grid caps of the grid-stride O(n) kernels);
// 1 if it cannot be read, which only narrows those grids.
inline int current_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 1;
    return sms;
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  The kernels of a leapfrog step (pack,
// offsets, force) and of a step of the adjoint sweep (reverse step, offsets,
// VJP) are launched so that each may be scheduled while its predecessor still
// runs: a chain kernel lets its successor launch as soon as it starts
// (pdl_trigger) and waits, in every CTA and before its first access to global
// memory that a kernel of the chain writes, until its predecessor has
// completed with its writes visible (pdl_wait).  Since every kernel of a
// chain waits that way before it can finish, each one completes only after
// all earlier ones, and a successor never reads or overwrites data an earlier
// kernel still uses.  (Before the wait a kernel may read what no kernel of
// the chain writes, such as the masses and the call's Morton permutation:
// those are complete before the chain's first kernel starts, and a chain
// kernel cannot start before that one.)  What this hides is the launch
// latency and CTA start-up between the short kernels of a step.  Outside such
// a launch both instructions do nothing.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Load of data that an earlier kernel of such a chain wrote, after pdl_wait.
// Through L2, the point of coherence (ld.global.cg): the read-only data path,
// which the compiler may pick for const __restrict__ pointers, gave stale
// values on GB300 once a kernel could start before its predecessor finished
// (a three-step leapfrog returned different bits from run to run, once off by
// 3e-5 in a velocity).  Every chain kernel reads its predecessors' results
// through this.
template <typename T>
__device__ __forceinline__ T ld_chain(const T* p) {
    return __ldcg(p);
}

// Off while kernels are timed one by one (profiling) or when NBODY_NO_PDL is set.
bool pdl_on();

// kernel<<<grid, block, smem, st>>>(args...), with programmatic serialisation
// against the preceding kernel of the stream when pdl_on().
template <typename... P, typename... A>
cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_on() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<A&&>(args)...);
}

// ---------------------------------------------------------------------------
// Host-side launch interfaces (implemented in force.cu / pack.cu / reduce.cu).
// ---------------------------------------------------------------------------
struct ForceShape {
    int threads;    // threads per CTA
    int ipairs;     // packed i-pairs per thread (2*ipairs bodies)
    int jtile;      // j-bodies per shared-memory stage
    int block;      // bodies per i-block = cell = 2*ipairs*threads
};

int force_num_shapes();
ForceShape force_shape(int k);

struct ForceArgs {
    const float* jdup;      // sources [npad][8]
    const double* centres;  // [nblk][3] cell centres (mixed) or nullptr (plain)
    float eps2;
    int64_t n;              // sinks
    int64_t npad;           // sources, padded to whole cells
    // Separate sinks (nullptr: the sinks are the sources, self pair masked).
    const float* ipack = nullptr;     // [nipad][8]
    const double* icentres = nullptr; // sink cell centres (mixed)
    int64_t nipad = 0;
    const int* perm = nullptr;        // sink slot k is body perm[k] (results go to perm[k])
    float* acc;             // [n][3]
    float* pot;             // [n] or nullptr
    double* partial;        // scratch, force_partial_doubles(...) doubles
    int* err;               // device error word
    int summation;          // 0 FP32 running sum, 1 per-tile Kahan fold, 2 Kahan per pair
    // Device word, nonzero when every source has the same mass (the kernel
    // then leaves m_j out of the pair loop and scales the sums once); nullptr:
    // treat the masses as distinct.
    const int* uni = nullptr;
};

// Scratch doubles needed for the split i-block partial sums of shape k.
size_t force_partial_doubles(int k, int num_sms);
// Adds the per-CTA partial sums (double4 per body: three vector components and
// one scalar) of every i-block a stream-K slice boundary cut (gpb = granules
// per i-block row, npad / kGranule), in CTA order, and
// writes out3[3g..3g+2] and out1[g] = -(scalar) for those blocks.
cudaError_t split_fixup(int64_t n, int64_t nblk, int64_t gpb, int64_t nctas, int block, const double* partial,
                        float* out3, float* out1, cudaStream_t st, const int* perm = nullptr,
                        int* err = nullptr);

// The partial sums of a force launch whose fixup was left to the next pack
// kernel: for the i-blocks a stream-K slice boundary cut, the pack adds the
// per-CTA partials itself (in CTA order, rounded to FP32 as the fixup does, so
// the result is the same bits) instead of reading the acceleration array.
struct SplitSums {
    const double* partial = nullptr;  // nullptr: every acceleration is in the acceleration array
    int64_t units = 0;                // granules of the launch
    int64_t nctas = 0;                // its CTAs
    int64_t gpb = 0;                  // granules per i-block row
    int block = 0;                    // bodies per i-block
};

// Exact scratch doubles force_launch needs for this variant and padded size
// (its grid: resident CTAs on num_sms SMs, capped by the work units).
size_t force_partial_doubles_for(int k, bool pot, bool mixed, bool compensated, int64_t npad, int num_sms);
// Launch the force kernel (stream-K over i-block x j-tile units) and the fixup
// that combines split i-blocks; *launched gets the number of kernels queued.
// ev0/ev1 (optional) are recorded on `st` just before and after the force
// kernel itself.  Returns a cudaError_t.
// With defer != nullptr the fixup is not launched and *defer describes the
// partial sums for the pack kernel that consumes them (sinks = sources only).
cudaError_t force_launch(int k, const ForceArgs& a, int num_sms, cudaStream_t st, int* launched,
                         cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr, SplitSums* defer = nullptr);

// Pack kernels: build jdup (and cell centres) from the state, optionally
// applying a kick (vel += kick * acc) and a drift (pos += drift * vel) first.
// All FP64 state arithmetic for the mixed path happens here.
// perm (optional): slot k of the packed array holds body perm[k].
int pack_threads(int block);
// *flag = 1 if mass[0..n) all compare equal, else 0.  Queues a memset
// and one kernel on st.
cudaError_t uniform_mass_flag(int64_t n, const float* mass, int* flag, cudaStream_t st);
// ss (optional): the accelerations of split i-blocks are in these deferred
// partial sums (see SplitSums) rather than in acc.  pack_f64 needs block to be
// a multiple of 256, and a centres buffer of pack_centre_doubles(npad, block)
// doubles (the cell centres, then the 256-body chunk sums); it queues
// pack_f64_launches(plain) kernels.
size_t pack_centre_doubles(int64_t npad, int block);
int pack_f64_launches(bool plain);
cudaError_t pack_f64(int64_t n, int64_t npad, int block, double* pos, double* vel, const float* acc,
                     const float* mass, double kick, double drift, bool plain, float* jdup,
                     double* centres, cudaStream_t st, const int* perm = nullptr, int* err = nullptr,
                     const SplitSums* ss = nullptr);
// The mixed-precision pack of a leapfrog step after the first of a call, in
// one kernel: each cell's centre is the mean of its bodies one step earlier,
// from the chunk sums (pack_chunk_doubles(npad) doubles) that the previous
// pack of the call wrote (pack_f64 writes them after the cell centres);
// the new positions' chunk sums go to chunks_out.  Needs vel and acc.
size_t pack_chunk_doubles(int64_t npad);
cudaError_t pack_f64_lagged(int64_t n, int64_t npad, int block, double* pos, double* vel, const float* acc,
                            const float* mass, double kick, double drift, float* jdup, double* centres,
                            const double* chunks_in, double* chunks_out, cudaStream_t st, const int* perm = nullptr,
                            int* err = nullptr, const SplitSums* ss = nullptr);
cudaError_t pack_f32(int64_t n, int64_t npad, float* pos, float* vel, const float* acc,
                     const float* mass, float kick, float drift, float* jdup, cudaStream_t st,
                     const SplitSums* ss = nullptr);

// vel += kick * acc (the closing half kick of a leapfrog call).
cudaError_t kick_f64(int64_t n, double* vel, const float* acc, double kick, cudaStream_t st);
cudaError_t kick_f32(int64_t n, float* vel, const float* acc, float kick, cudaStream_t st);

// FP64 diagnostics reduction: out9 (device, 9 doubles) = T, W, E, P[3], F[3].
// `scratch` holds reduce_scratch_doubles() doubles.
size_t reduce_scratch_doubles();
cudaError_t energy_reduce_f64(int64_t n, const double* vel, const float* mass, const float* acc,
                              const float* pot, double* scratch, double* out9, cudaStream_t st);
cudaError_t energy_reduce_f32(int64_t n, const float* vel, const float* mass, const float* acc,
                              const float* pot, double* scratch, double* out9, cudaStream_t st);

// ---- ragged batches (batched.cu) ----
struct BatchShape {
    int threads;  // threads per CTA
    int ibodies;  // i-bodies per thread per pass
};
struct BatchArgs {
    int64_t nsys;
    const int64_t* offsets;  // device [nsys+1]
    const float* eps;        // device [nsys]
    float* pos;
    float* vel;
    const float* mass;
    float* acc;
    float* pot;
    float dt;
    int64_t steps;  // 0: force only (acc, pot); > 0: leapfrog in place
    int cap;        // bodies of the shared-memory image; larger systems take the multi-CTA path
    bool coop;      // a system may exceed cap: cooperative launch, full resident grid
    void* scratch;  // batched_scratch_bytes(nsys) bytes (plan, order, barriers)
    int* err;       // error word
};
int batched_num_shapes();
BatchShape batched_shape(int k);
size_t batched_smem_bytes(int cap);
size_t batched_scratch_bytes(int64_t nsys);
// Shared-memory image (bodies, a multiple of 128) a CTA of shape k gets when
// the batch's sizes are not known on the host: as large as the resident CTAs
// its registers allow per SM can each have.
int batched_max_cap(int k);
// Queues the planning kernels and the persistent kernel; *launched gets the
// number of kernels queued.
cudaError_t batched_launch(int k, const BatchArgs& a, int num_sms, cudaStream_t st, int* launched);

// ---- reverse mode (vjp.cu) ----
struct VjpShape {
    int threads;
    int ipairs;
    int jtile;
    int block;
};
struct VjpArgs {
    const float* jv;        // [npad][16] (pack_vjp)
    const double* centres;  // [nblk][3] or nullptr (plain)
    float eps2;
    int64_t n;
    int64_t npad;
    bool has_mu;            // potential cotangent present
    float* g_pos;           // [n][3]
    float* g_mass;          // [n]
    float* acc = nullptr;   // [n][3]: also the force at the same positions (no potential cotangent)
    double* partial;
    int* err;
    // Device word, nonzero when every body has the same mass (the pair loop
    // then forms u = mu (lam_j - lam_k) without the masses); nullptr: no.
    const int* uni = nullptr;
};
int vjp_num_shapes();
VjpShape vjp_shape(int k);
int vjp_floats_per_body();
size_t vjp_partial_doubles(int k, int num_sms);
// Pack the VJP j-array.  With lam_f64/lamx given (adjoint sweep) it first does
// lamx += gprev, gm_acc += gmprev, lam_f64 += drift * lamx; the cotangent
// packed is kappa * lam.
// One step of the leapfrog run backwards, done by pack_vjp before it packs
// (the adjoint sweep's positions without a forward replay):
//   vh -= kick * a;  x -= drift * vh
// with a the force at the previous positions (from acc, or from its deferred
// partial sums ss_acc); or, at a checkpoint, x and vh taken from the tape.
struct ReverseStep {
    double* x = nullptr;              // positions [n][3], updated in place; nullptr: no reverse step
    double* vh = nullptr;             // half-step velocities [n][3], updated in place
    const double* anchor_x = nullptr; // checkpoint: x and vh are copied from here (kick, drift ignored)
    const double* anchor_v = nullptr;
    const float* a = nullptr;         // force at the previous positions, [n][3]; nullptr: no kick
    SplitSums ss_acc;                 // its deferred partial sums
    double kick = 0.0;
    double drift = 0.0;
};

// Two kernels; centres holds pack_centre_doubles(npad, block) doubles (block a
// multiple of 256).  ss (optional): g_prev/gm_prev of split i-blocks are in the
// previous VJP's deferred partial sums.  rev (optional): the reverse step,
// after which pos is rev->x.
cudaError_t pack_vjp(int64_t n, int64_t npad, int block, const double* pos, const float* mass, const float* lam_f32,
                     double* lam_f64, double* lamx, const float* gprev, const float* gmprev, double* gm_acc,
                     double drift, double kappa, const float* mu, bool plain, float* jv, double* centres,
                     cudaStream_t st, const SplitSums* ss = nullptr, const ReverseStep* rev = nullptr);
// The adjoint sweep's pack after its first, in one kernel (mixed precision;
// lam_f64, lamx and rev->x required): as pack_vjp, with each cell's centre
// the mean of its bodies one step earlier, from the chunk sums
// (pack_chunk_doubles(npad) doubles) the previous pack left in chunks_in
// (pack_vjp writes them after the cell centres); the new positions' chunk
// sums go to chunks_out.
cudaError_t pack_vjp_lagged(int64_t n, int64_t npad, int block, const float* mass, double* lam_f64, double* lamx,
                            const float* gprev, const float* gmprev, double* gm_acc, double drift, double kappa,
                            float* jv, double* centres, const double* chunks_in, double* chunks_out,
                            cudaStream_t st, const SplitSums* ss, const ReverseStep* rev);
cudaError_t adjoint_accumulate(int64_t n, double* lamx, const float* g, double* gm_acc, const float* gm,
                               cudaStream_t st);
// ev0/ev1 (optional) are recorded on `st` just before and after the VJP kernel.
// defer (optional): skip the fixup; the next pack_vjp adds the partials.
// defer_acc (optional, with a.acc): the same for the force.
cudaError_t vjp_launch(int k, const VjpArgs& a, int num_sms, cudaStream_t st, int* launched,
                       cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr, SplitSums* defer = nullptr,
                       SplitSums* defer_acc = nullptr);

// ---- spatial order (order.cu) ----
// perm[k] = index of the body at position k of the Morton order (stable, by
// index within equal keys).  `scratch` holds order_scratch_bytes(n) bytes.
size_t order_scratch_bytes(int64_t n);
cudaError_t spatial_order(int64_t n, const double* pos, int* perm, void* scratch, cudaStream_t st);
// One stable pass of the same radix sort: (key_out, val_out) = (key_in, val_in)
// ordered by the 8-bit digit (key >> shift) & 255, ties in index order.
// `hist` holds sort_pass_hist_ints(n) ints.  Three kernels on st.
size_t sort_pass_hist_ints(int64_t n);
cudaError_t sort_pass(int64_t n, const unsigned* key_in, const int* val_in, int shift, unsigned* key_out,
                      int* val_out, int* hist, cudaStream_t st);

// One CTA waits on an mbarrier nothing completes, for limit_ns, then sets *err.
cudaError_t selftest_wait(uint64_t limit_ns, int* err, cudaStream_t st);

// The CTAs of a stream-K launch whose slices touch i-block b: [*c_lo, *c_hi],
// and the partial slot c_lo wrote (0 if its slice starts at the block, else 1;
// every later CTA starts inside the block, slot 0).
__host__ __device__ __forceinline__ void split_ctas(int64_t b, int64_t gpb, int64_t units, int64_t nctas,
                                                    int64_t* c_lo, int64_t* c_hi, int* slot_lo) {
    const int64_t u0 = b * gpb, u1 = u0 + gpb - 1;
    *c_lo = ((u0 + 1) * nctas - 1) / units;
    *c_hi = ((u1 + 1) * nctas - 1) / units;
    *slot_lo = (*c_lo * units / nctas == u0) ? 0 : 1;
}

// Partial sums of split i-blocks in double-float: each component is the
// unevaluated sum hi + lo of two FP32 values (about 48 significant bits), so
// forming, scaling and adding partials takes FP32 instructions only.  On
// GB300 the FP64 pipe runs at about 1/64 of the FP32 rate: the FP64 epilogue
// and partial sums these replace held the FP64 pipe for several microseconds
// of every mid-size force launch.
struct DF {
    float hi, lo;
};
// a + b exactly (Knuth's two-sum): s = fl(a + b), e the rounding error.
__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return DF{s, (a - (s - bb)) + (b - bb)};
}
// a + b, renormalised (|lo| at most half an ulp of hi).
__device__ __forceinline__ DF df_add(DF a, DF b) {
    const DF s = two_sum(a.hi, b.hi);
    const float lo = s.lo + (a.lo + b.lo);
    const float hi = s.hi + lo;
    return DF{hi, lo - (hi - s.hi)};
}
// a * m, renormalised (the product's rounding error recovered with an FMA).
__device__ __forceinline__ DF df_scale(DF a, float m) {
    const float p = a.hi * m;
    const float lo = fmaf(a.lo, m, fmaf(a.hi, m, -p));
    const float hi = p + lo;
    return DF{hi, lo - (hi - p)};
}
__device__ __forceinline__ float df_float(DF a) { return a.hi + a.lo; }

// One partial record: four double-float components (x, y, z, w), 32 bytes,
// in the buffers sized in doubles (four per record).
__device__ __forceinline__ double df_bits(DF a) {
    return __hiloint2double(__float_as_int(a.lo), __float_as_int(a.hi));  // hi in the low word
}
__device__ __forceinline__ void store_partial(double* partial, int64_t rec, DF x, DF y, DF z, DF w) {
    reinterpret_cast<double4_16a*>(partial)[rec] = make_double4_16a(df_bits(x), df_bits(y), df_bits(z), df_bits(w));
}

// Sum in CTA order of the partial records of slot lb of block b, rounded to
// FP32 at the end.  NB loads are issued before the first is added (a block of
// a mid-size launch has ~20 CTAs' partials: one or a few rounds of L2 latency
// instead of twenty); the additions keep CTA order whatever NB is, so every
// NB gives the same bits.  W: also the fourth component (the potential, or
// the VJP's mass gradient); without it s4[3] is left alone and each record's
// last 8 bytes are not read.
template <int NB = 8, bool W = true>
__device__ __forceinline__ void split_sum(const double* partial, int C, int64_t b, int64_t c_lo, int64_t c_hi,
                                          int slot_lo, int lb, float* s4) {
    const float4* P = reinterpret_cast<const float4*>(partial);
    const float2* P2 = reinterpret_cast<const float2*>(partial);
    DF sx{0.0f, 0.0f}, sy{0.0f, 0.0f}, sz{0.0f, 0.0f}, sw{0.0f, 0.0f};
    for (int64_t c0 = c_lo; c0 <= c_hi; c0 += NB) {
        float4 v0[NB], v1[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int64_t c = c0 + q;
            if (c <= c_hi) {
                const int64_t rec = (c * 2 + (c == c_lo ? slot_lo : 0)) * C + lb;
                v0[q] = ld_chain(P + 2 * rec);
                if (W) {
                    v1[q] = ld_chain(P + 2 * rec + 1);
                } else {
                    const float2 z = ld_chain(P2 + 4 * rec + 2);
                    v1[q] = make_float4(z.x, z.y, 0.0f, 0.0f);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            if (c0 + q <= c_hi) {
                sx = df_add(sx, DF{v0[q].x, v0[q].y});
                sy = df_add(sy, DF{v0[q].z, v0[q].w});
                sz = df_add(sz, DF{v1[q].x, v1[q].y});
                if (W) sw = df_add(sw, DF{v1[q].z, v1[q].w});
            }
        }
    }
    s4[0] = df_float(sx);
    s4[1] = df_float(sy);
    s4[2] = df_float(sz);
    if (W) s4[3] = df_float(sw);
    (void)b;
}

// The split of the i-block holding slots [k0, k0 + 256) (one block: blocks are
// multiples of 256), computed by thread 0 and shared through shared memory
// (64-bit divisions are slow on the GPU; once per CTA, not per body).
// Every thread of the CTA must call it.
struct BlockSplit {
    int64_t b, c_lo, c_hi;
    int slot_lo;
};
__device__ __forceinline__ BlockSplit block_split(const SplitSums& ss, int64_t k0) {
    __shared__ BlockSplit sh;
    if (threadIdx.x == 0) {
        BlockSplit r{0, 0, 0, 0};
        if (ss.partial != nullptr) {
            r.b = k0 / ss.block;
            split_ctas(r.b, ss.gpb, ss.units, ss.nctas, &r.c_lo, &r.c_hi, &r.slot_lo);
        }
        sh = r;
    }
    __syncthreads();
    return sh;
}

// The acceleration of slot k (body g): from the deferred partial sums of its
// block when the block was split, else from acc.  NB: loads in flight (see
// split_sum).
template <int NB = 8>
__device__ __forceinline__ void split_acc(const SplitSums& ss, const BlockSplit& bs, int64_t k, int64_t g,
                                          const float* acc, float* out) {
    if (ss.partial != nullptr && bs.c_lo < bs.c_hi) {
        float s4[4];
        split_sum<NB, false>(ss.partial, ss.block, bs.b, bs.c_lo, bs.c_hi, bs.slot_lo, (int)(k - bs.b * ss.block),
                             s4);
        out[0] = s4[0];
        out[1] = s4[1];
        out[2] = s4[2];
        return;
    }
    out[0] = ld_chain(acc + 3 * g + 0);
    out[1] = ld_chain(acc + 3 * g + 1);
    out[2] = ld_chain(acc + 3 * g + 2);
}

}  // namespace nbk
