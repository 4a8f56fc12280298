/*
 * nbody.h -- C ABI of libnbody: all-pairs Plummer-softened gravity on one
 * NVIDIA GB300 (sm_103a), with a kick-drift-kick leapfrog driven by it.
 *
 * The operation is the N-body demonstration of Miki & Hanawa, "Unified
 * schemes for directive-based GPU offloading" (IEEE Access 2024), Sec. III.A:
 *
 *   Eq. 1 (G = 1, Henon units):
 *     a_i = sum_{j != i} m_j (r_j - r_i) / (|r_j - r_i|^2 + eps^2)^{3/2}
 *   and the potential that Listing 4 accumulates under CALCULATE_POTENTIAL,
 *   returned with the physical sign and without the self term:
 *     phi_i = -sum_{j != i} m_j / (|r_j - r_i|^2 + eps^2)^{1/2}
 *
 * Listing 4's calc_acc(Ni, ipos, iacc, Nj, jpos, eps) fixes the per-pair
 * arithmetic these kernels keep: r2 as an FMA chain seeded with eps^2, an
 * approximate reciprocal square root cubed and scaled by m_j, FMA
 * accumulation, single precision with flush-to-zero (Sec. III.A notes that
 * fast approximate rsqrt is essential to performance).
 *
 * Conventions shared by every call:
 *  - Arrays are contiguous: positions, velocities and accelerations are
 *    array-of-structures [n][3]; mass and potential are [n].
 *  - A pointer may address device memory or host memory (pageable or pinned).
 *    Device arrays are used in place and the call is asynchronous on
 *    opts->stream; results are valid once that stream has synchronised.
 *    If any array of a call is in host memory, the library copies the host
 *    arrays through its device workspace and the call returns only after the
 *    results are back in host memory.
 *  - The caller owns every array; the library never frees or keeps them past
 *    the call.  Internal workspace is cached per (device, stream) and freed by
 *    nbody_finalize().  Calls on the same stream are ordered; calls on
 *    different streams use different workspaces.
 *  - The current CUDA device of the calling thread is used.
 *  - Return value: NBODY_OK (0) or one of the negative codes below.
 *    n == 0 is a no-op returning NBODY_OK.  Arguments are validated before
 *    any GPU work is queued (NBODY_EINVAL: n < 0, a required pointer NULL,
 *    eps < 0 or not finite, dt not finite, steps < 0).
 *  - Coincident bodies with eps == 0 give non-finite results, as Eq. 1 does;
 *    the self pair is always excluded exactly, so eps == 0 is valid for
 *    distinct positions.
 *  - Interactions are counted as n*n per force evaluation (the paper's
 *    "interaction pairs", Sec. III.A).
 *  - When every source mass is equal (checked on the device at the start of
 *    each call) the force and VJP kernels leave the mass out of the pair loop
 *    and scale the sums by it once: the same result to FP32 rounding, one
 *    operation fewer per interaction.
 *  - Each call opens an NVTX range named after it (visible to timeline
 *    tools; a no-op otherwise).
 *  - Environment: NBODY_TUNE_FILE names the kernel-shape table (default:
 *    nbody_tune.txt beside the library); NBODY_NO_GRAPH turns off the graph
 *    replay of repeated calls; NBODY_FAULT=alloc|launch|tune injects a
 *    host-side failure for tests (NBODY_ENOMEM, NBODY_ECUDA, an unreadable
 *    shape table) without queuing GPU work.
 */
#ifndef NBODY_H
#define NBODY_H

#include <stdint.h>

#if defined(__GNUC__)
#define NBODY_API __attribute__((visibility("default")))
#else
#define NBODY_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define NBODY_OK 0
#define NBODY_EINVAL (-1)   /* invalid argument */
#define NBODY_ENOMEM (-2)   /* device or pinned memory allocation failed */
#define NBODY_ECUDA (-3)    /* a CUDA runtime call failed; see nbody_last_cuda_error() */
#define NBODY_ETIMEOUT (-4) /* a bounded device-side wait expired (kernel returned early) */
#define NBODY_ENOTSUP (-5)  /* no usable sm_103 device or unsupported option */
#define NBODY_EBOUNDS (-6)  /* a kernel of a checked build (-DNBODY_CHECKS) met an index out of range */

/* Pair arithmetic precision. */
#define NBODY_PREC_MIXED 0 /* FP64 positions; FP32 pair math on coordinates
                              relative to the FP64 centres of cells of
                              bodies sorted along a Morton curve (default) */
#define NBODY_PREC_PLAIN 1 /* FP32 absolute coordinates (FP64 input rounded) */
#define NBODY_PREC_MIXED_UNSORTED 2 /* mixed, with cells taken in the caller's
                                       order instead of a Morton order */

/* Per-body summation over j. */
#define NBODY_ACC_COMPENSATED 0 /* FP32 per j-tile, tiles folded by Kahan
                                   summation (default) */
#define NBODY_ACC_FP32 1        /* one running FP32 sum over all j */
#define NBODY_ACC_KAHAN_PAIR 2  /* Kahan summation of every pair term: the most
                                   accurate and about twice the FP32 work */

typedef struct nbody_opts {
    void* stream;   /* cudaStream_t to run on; NULL = legacy default stream */
    int precision;  /* NBODY_PREC_*; ignored by the *_f32 calls (always plain) */
    int accumulate; /* NBODY_ACC_* */
    int config;     /* force-kernel shape index, -1 = the tuned choice for n;
                       valid indices are 0 .. nbody_num_configs()-1 */
    int reserved;   /* must be 0 */
} nbody_opts;

/* Fill *opts with the defaults (NULL stream, mixed, compensated, tuned). */
NBODY_API void nbody_opts_default(nbody_opts* opts);

/*
 * Acceleration (Eq. 1) and potential for all n bodies, FP64 positions.
 *  pos  [n][3] double, mass [n] float, eps >= 0
 *  acc  [n][3] float, written
 *  pot  [n] float or NULL (NULL skips the potential term, a cheaper kernel)
 * opts->precision selects mixed (default) or plain FP32 coordinates.
 */
NBODY_API int nbody_accel(int64_t n, const double* pos, const float* mass, double eps, float* acc, float* pot,
                const nbody_opts* opts);

/* The same with FP32 positions and softening (plain precision, Listing 4's
 * data types). */
NBODY_API int nbody_accel_f32(int64_t n, const float* pos, const float* mass, float eps, float* acc, float* pot,
                    const nbody_opts* opts);

/*
 * Kick-drift-kick leapfrog driven by Eq. 1, in place (not in the paper; the
 * integrator the demonstration's force evaluation drives):
 *   v += (dt/2) a(x);  x += dt v;  v += (dt/2) a(x)      (per step)
 * The force at the end of a step serves the first kick of the next, so a call
 * makes steps + 1 force evaluations.  pos, vel [n][3] double (FP64 drift and
 * kicks), mass [n] float.  steps == 0 leaves the state unchanged.
 *
 * A call repeated with the same arguments (device arrays, same stream and
 * options: a simulation loop) is captured into a CUDA graph on its second
 * occurrence and replayed as one unit from then on, with results
 * bit-identical to direct launches; nbody_leapfrog_batched does the same.
 * Graphs are not used while profiling is on (nbody_profile_enable), when the
 * environment sets NBODY_NO_GRAPH, or when a CUDA tool is injected into the
 * process (CUDA_INJECTION64_PATH set, as under ncu), so tools see every
 * kernel launched directly.
 */
NBODY_API int nbody_leapfrog(int64_t n, double* pos, double* vel, const float* mass, double eps, double dt,
                   int64_t steps, const nbody_opts* opts);

/* The same with FP32 state (plain precision). */
NBODY_API int nbody_leapfrog_f32(int64_t n, float* pos, float* vel, const float* mass, float eps, float dt,
                       int64_t steps, const nbody_opts* opts);

/*
 * Diagnostics, reduced in FP64 on the device (synchronous; out is host memory):
 *  out[0] T = sum m|v|^2/2, out[1] W = (1/2) sum m_i phi_i, out[2] E = T + W,
 *  out[3..5] momentum sum m v, out[6..8] net force sum m a (zero by Newton's
 *  third law up to rounding).  One force-and-potential evaluation.
 */
NBODY_API int nbody_energy(int64_t n, const double* pos, const double* vel, const float* mass, double eps,
                 double* out, const nbody_opts* opts);
NBODY_API int nbody_energy_f32(int64_t n, const float* pos, const float* vel, const float* mass, float eps,
                     double* out, const nbody_opts* opts);

/*
 * Ragged batches: nsys independent systems in one persistent launch.  System s
 * owns bodies [offsets[s], offsets[s+1]) of the concatenated arrays; each has
 * its own softening eps[s] and interacts only with itself (Eq. 1 per system).
 *  offsets [nsys+1] int64: offsets[0] == 0, non-decreasing, every system below
 *          2^31 bodies; any system size is accepted.  A system that fits one
 *          CTA's shared memory (about 14,000 bodies on GB300) is owned by one
 *          CTA for the whole call; a larger one is split over several CTAs
 *          that stream its bodies through shared memory and meet at a
 *          barrier of their own between the phases of each step.
 *  pos [N][3] float, mass [N] float, eps [nsys] float (>= 0, finite)
 *  acc [N][3] float written; pot [N] float or NULL.
 * Offsets and softenings in device memory are checked on the device: the
 * call returns at once (asynchronous like every call on device arrays) and a
 * bad batch is skipped, nothing written, and reported as NBODY_EINVAL by
 * nbody_last_device_error().  Those in host memory are checked on the host
 * (NBODY_EINVAL before any work is queued).  The largest-first order of the
 * systems is computed on the device in both cases.
 * FP32 state and pair arithmetic; per-body sums in two levels (64-pair
 * blocks), plus a Kahan fold per tile for systems split over several CTAs.
 * opts->config selects the batched kernel shape (0 .. nbody_num_batched_configs()-1:
 * threads per CTA, i-slots per warp, j-loop unroll and the depth of the FP32
 * j-blocks differ), -1 = the tuned
 * choice for the largest system when the offsets are host memory, else 0;
 * precision and accumulate are ignored.
 */
NBODY_API int nbody_accel_batched(int64_t nsys, const int64_t* offsets, const float* pos, const float* mass,
                                  const float* eps, float* acc, float* pot, const nbody_opts* opts);

/* Kick-drift-kick leapfrog of every system of a ragged batch, all steps inside
 * one persistent kernel (steps + 1 force evaluations per system); pos, vel
 * [N][3] float updated in place, dt rounded to FP32 for the FP32 state. */
NBODY_API int nbody_leapfrog_batched(int64_t nsys, const int64_t* offsets, float* pos, float* vel,
                                     const float* mass, const float* eps, double dt, int64_t steps,
                                     const nbody_opts* opts);

/*
 * Separate sinks and sources: Listing 4's own form calc_acc(Ni, ipos, iacc,
 * Nj, jpos, eps).  acc[i] = sum_j m_j (r_j - r_i) / (|r_j - r_i|^2 + eps^2)^{3/2}
 * and pot[i] = -sum_j m_j / (|r_j - r_i|^2 + eps^2)^{1/2} over all ni sinks and
 * all nj sources, every pair included (a sink that coincides with a source
 * gets zero force from it when eps > 0, -m_j/eps of potential, and a
 * non-finite result when eps == 0).  Useful for subsample evaluation and for
 * splitting the sinks of one system over several devices.
 *  ipos [ni][3], jpos [nj][3] (double, or float for the _f32 call),
 *  jmass [nj] float, acc [ni][3] float, pot [ni] float or NULL.
 * nj == 0 writes zeros; mixed precision as nbody_accel (the _f32 call is plain).
 */
NBODY_API int nbody_accel_ij(int64_t ni, const double* ipos, int64_t nj, const double* jpos, const float* jmass,
                             double eps, float* acc, float* pot, const nbody_opts* opts);
NBODY_API int nbody_accel_ij_f32(int64_t ni, const float* ipos, int64_t nj, const float* jpos, const float* jmass,
                                 float eps, float* acc, float* pot, const nbody_opts* opts);

/*
 * Reverse mode of Eq. 1 (not in the paper; the derivative of the force it
 * defines).  For cotangents g_acc of the accelerations and g_pot of the
 * potentials (NULL = none), with d = r_j - r_k, s = |d|^2 + eps^2 and the tidal
 * tensor T(d) = s^{-3/2} I - 3 s^{-5/2} d d^T:
 *   g_pos[k]  = sum_{j != k} T(d) (m_k g_acc[j] - m_j g_acc[k])
 *               - sum_{j != k} s^{-3/2} d (g_pot[j] m_k + g_pot[k] m_j)
 *   g_mass[k] = -sum_{j != k} [ s^{-3/2} (g_acc[j] . d) + g_pot[j] s^{-1/2} ]
 * i.e. the gradients of sum_i g_acc[i].a_i + g_pot[i] phi_i.  A second
 * all-pairs pass (30 FP32 operations per pair); mixed precision as nbody_accel.
 *  pos [n][3] double, mass [n] float, g_acc [n][3] float, g_pot [n] float or
 *  NULL; g_pos [n][3] float and g_mass [n] float are overwritten.
 * opts->config selects the VJP kernel shape (0 .. 3), -1 = default.
 */
NBODY_API int nbody_accel_vjp(int64_t n, const double* pos, const float* mass, double eps, const float* g_acc,
                    const float* g_pot, float* g_pos, float* g_mass, const nbody_opts* opts);

/*
 * Differentiating a leapfrog trajectory, checkpointed (not in the paper; the
 * exact discrete adjoint of the kick-drift-kick steps nbody_leapfrog takes).
 *
 * nbody_leapfrog_vjp: for cotangents g_posT = dL/dx(T) and g_velT = dL/dv(T)
 * of a run of `steps` steps from pos0, vel0, returns the gradients
 * dL/dx(0), dL/dv(0) and the dynamics' part of dL/dm (FP64; a loss that also
 * depends on m directly adds its own term).  pos0, vel0 [n][3] double and
 * mass [n] float are inputs only (the run is recorded on copies in the
 * library's workspace, with checkpoints every ckpt_every steps); every array
 * may be host or device memory.  Cost: one forward run plus the sweep below.
 *
 * The same in two calls, for a caller that makes the forward run anyway:
 * nbody_leapfrog_record runs nbody_leapfrog (FP64 state, in place) and writes
 * a tape: for every checkpoint step k = 0, c, 2c, ... < steps (c = ckpt_every)
 * the positions x_k and half-step velocities v_{k+1/2}, then x_steps and
 * v_{steps-1/2} (nbody_tape_bytes(n, steps, c) bytes of device memory,
 * caller-owned).  nbody_leapfrog_vjp_tape is the reverse sweep from that
 * tape: one force VJP per force evaluation of the forward run, newest first,
 * at positions obtained by running the leapfrog backwards from the end
 * (x_s = x_{s+1} - dt v_{s+1/2}, v_{s-1/2} = v_{s+1/2} - dt a(x_s), the
 * force computed by the VJP kernel itself at x_s) and reset to the recorded
 * state at every checkpoint -- so no forward replay, and a reversed state is
 * at most c - 1 steps from a recorded one (they agree to rounding).  The tape
 * and mass must be device memory; the cotangent and gradient arrays may be
 * host or device.  nbody_tape_bytes returns -1 for invalid sizes.
 */
NBODY_API int nbody_leapfrog_vjp(int64_t n, const double* pos0, const double* vel0, const float* mass, double eps,
                                 double dt, int64_t steps, int64_t ckpt_every, const double* g_posT,
                                 const double* g_velT, double* g_pos0, double* g_vel0, double* g_mass,
                                 const nbody_opts* opts);
NBODY_API int64_t nbody_tape_bytes(int64_t n, int64_t steps, int64_t ckpt_every);
NBODY_API int nbody_leapfrog_record(int64_t n, double* pos, double* vel, const float* mass, double eps, double dt,
                                    int64_t steps, int64_t ckpt_every, void* tape, const nbody_opts* opts);
NBODY_API int nbody_leapfrog_vjp_tape(int64_t n, const float* mass, double eps, double dt, int64_t steps,
                                      int64_t ckpt_every, const void* tape, const double* g_posT,
                                      const double* g_velT, double* g_pos0, double* g_vel0, double* g_mass,
                                      const nbody_opts* opts);

/* Number of force-kernel shapes compiled in (for opts->config) and the
 * bodies per i-block of shape k (0 if k is out of range). */
NBODY_API int nbody_num_configs(void);
NBODY_API int nbody_config_block(int k);
/* Number of batched-kernel shapes compiled in (opts->config of the batched
 * calls). */
NBODY_API int nbody_num_batched_configs(void);

/*
 * Kernel-shape table (the paper chose its thread count by a parameter survey
 * on each machine, Sec. III.A; paper_2411_18889_gb300.tune runs that survey
 * and writes the table).  nbody_tune_load(path) replaces the rules with those
 * of a file (path NULL: NBODY_TUNE_FILE, else nbody_tune.txt beside the
 * library, else the built-in GB300 table) and returns the number of rules or
 * NBODY_EINVAL (malformed line or shape index out of range; the table is then
 * unchanged).  Lines: "force <pot 0|1> <n_min> <shape>", "vjp <n_min>
 * <shape>", "batched [<n_min>] <shape>" (for a batched rule n_min is compared
 * with the largest system of the batch; omitted, it is 0), '#' comments; the
 * rule of a kind with the largest n_min <= n applies.  nbody_tuned_shape(kind, n, pot)
 * returns the shape used for kind 0 (force), 1 (VJP) or 2 (batched; n = the
 * largest system) when opts->config is -1.
 */
NBODY_API int nbody_tune_load(const char* path);
NBODY_API int nbody_tuned_shape(int kind, int64_t n, int pot);

/* Synchronise the current device and report whether any kernel since the
 * last call hit a bounded-wait timeout (NBODY_ETIMEOUT), found a ragged
 * batch's device offsets or softenings invalid (NBODY_EINVAL; that batch was
 * skipped) or, in a checked build, an index out of range (NBODY_EBOUNDS; the
 * access was skipped) -- the flag is then cleared -- or a CUDA error
 * (NBODY_ECUDA); NBODY_OK otherwise. */
NBODY_API int nbody_last_device_error(void);

/* The last CUDA runtime error code seen by the library on this thread. */
NBODY_API int nbody_last_cuda_error(void);

/* Static description of an NBODY_* code. */
NBODY_API const char* nbody_strerror(int code);

/* Self-test of the bounded device-side wait that every pipelined kernel
 * uses: one CTA waits on a barrier phase that nothing completes, gives up
 * after limit_seconds (1e-6 .. 1), records the timeout and returns.
 * Synchronous; returns NBODY_ETIMEOUT when the timeout path works (the
 * GPU stays usable), NBODY_EINVAL for a limit out of range. */
NBODY_API int nbody_selftest_wait(double limit_seconds, const nbody_opts* opts);

/*
 * nbody_accel_noalloc -- nbody_accel with its default options (mixed
 * precision on cells of bodies in Morton order, compensated sums) and kernel
 * shape 1 (opts->config = 1), the potential when pot != NULL, for callers that
 * cannot allocate GPU memory.  Its results are bit-identical to that
 * nbody_accel call's.
 * The paper has no counterpart; this is a deployment variant of the same
 * force evaluation.
 *
 * Who needs it: code running where cudaMalloc is not allowed or not safe --
 * inside another framework's allocator or memory-pool callback, in a
 * real-time loop that must never wait on the driver's allocator, or in a
 * process that has reserved all device memory up front.  nbody_accel grows a
 * cached workspace with cudaMalloc; this call never allocates or frees
 * anything (no cudaMalloc, cudaFree or allocating library routine).
 *
 * Its scratch is one fixed array in the library's device module,
 * 24,453,376 bytes (23.3 MiB), which every GPU that loads the library holds
 * until the process exits.  Limits: n <= NBODY_NOALLOC_MAX_N (65536); larger n returns
 * NBODY_EINVAL without queuing work.  If the device needs more partial-sum
 * scratch than the array holds (a GPU with more SMs than it was sized for),
 * the call returns NBODY_ENOMEM.
 *
 *  pos [n][3] double, mass [n] float, acc [n][3] float (written), pot [n]
 *  float or NULL: device (or managed) memory only -- host arrays would need
 *  staging buffers, so they return NBODY_EINVAL.
 *  status: NULL, or a device int the call sets to 0 and its kernels set to 1
 *  if a bounded device-side wait expired (results then incomplete), or to 2
 *  in a checked build (-DNBODY_CHECKS) if an index was out of range.
 *  stream: cudaStream_t to run on (NULL = legacy default stream); the call
 *  is asynchronous.
 *
 * The first call on each device performs the set-up: it looks up the
 * device address of the scratch array (cudaGetSymbolAddress, with that
 * device current), which can load the library's device module.  Make that
 * first call before any stream capture.  Every call shares the one array and
 * it keeps the last call's contents, so calls that overlap on the GPU (two
 * streams, or two host threads without ordering) race and corrupt each
 * other: order them on one stream or synchronise between them.
 */
#define NBODY_NOALLOC_MAX_N 65536
NBODY_API int nbody_accel_noalloc(int64_t n, const double* pos, const float* mass, double eps, float* acc, float* pot,
                        int* status, void* stream);

/* Benchmark instrumentation.  While enabled, every force-kernel launch is
 * bracketed by a pair of CUDA events recorded on its own stream.
 * nbody_profile_read waits for those events and returns the summed device
 * time of the force kernels (ms) and their number since the previous read,
 * plus the number of kernels of every kind the library queued; then resets.
 * The leapfrog's integrator kernels are timed the same way:
 * nbody_profile_read_kind(kind, &ms, &launches) returns and resets the summed
 * device time and launch count of kind 0 (force kernel), 1 (pack kernel:
 * kick, drift and the packed j-array), 2 (closing kick kernel) or 3 (force
 * VJP kernel); NBODY_EINVAL for another kind. */
NBODY_API void nbody_profile_enable(int on);
NBODY_API int nbody_profile_read(double* force_ms, int64_t* force_launches, int64_t* all_launches);
NBODY_API int nbody_profile_read_kind(int kind, double* ms, int64_t* launches);

/* Free every cached workspace on every device (synchronises each device). */
NBODY_API void nbody_finalize(void);

/* Library version, major*10000 + minor*100 + patch. */
NBODY_API int nbody_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NBODY_H */
