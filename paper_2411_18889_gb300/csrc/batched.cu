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

#include "batched_kernel.cuh"

namespace nbk {
namespace {

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

struct BShapeEntry {
    BatchShape shape;
    BFn fn[2];  // [pot]
};

const BShapeEntry* bshapes() {
    static const BShapeEntry table[kNumBShapes] = {
        {{kBShapes[0].threads, kBShapes[0].ibodies}, {batched_fn_00(), batched_fn_01()}},
        {{kBShapes[1].threads, kBShapes[1].ibodies}, {batched_fn_10(), batched_fn_11()}},
        {{kBShapes[2].threads, kBShapes[2].ibodies}, {batched_fn_20(), batched_fn_21()}},
        {{kBShapes[3].threads, kBShapes[3].ibodies}, {batched_fn_30(), batched_fn_31()}},
        {{kBShapes[4].threads, kBShapes[4].ibodies}, {batched_fn_40(), batched_fn_41()}},
        {{kBShapes[5].threads, kBShapes[5].ibodies}, {batched_fn_50(), batched_fn_51()}},
    };
    return table;
}

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
