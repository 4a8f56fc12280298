// force.cu -- the all-pairs softened force and potential (Eq. 1 of Miki &
// Hanawa, Sec. III.A, with the per-pair arithmetic of their Listing 4).
//
// Occupancy.  The persistent grid holds 16 warps per SM (two 256-thread CTAs
// or one of 512) even when registers would allow more: with the FP32 FMA pipe
// as the bound, more resident warps only trade registers (ILP) for latency
// hiding the kernel does not need; on GB300 a 256-thread shape ran at 60.5 %
// of FP32 peak with three CTAs per SM and 66 % with two.
//
// Decomposition.  Bodies are grouped in i-blocks ("cells") of
// block = 2 * IP * T bodies; the j-range is cut into tiles of J bodies, and
// each tile into granules of 32 j-bodies.  The work is the grid of granules
// (i-block, 32 j-bodies), flattened i-block-major, and a persistent grid of P
// CTAs takes equal contiguous slices of it ("stream-K"): CTA c owns granules
// [c*U/P, (c+1)*U/P), so every CTA gets the same number of pair interactions
// to within one granule whatever n is, with no tail wave (with whole tiles as
// the unit, N = 16384 gave CTAs 6 or 7 tiles each: a 14 % spread).  The first
// and last tile of a slice may be used in part.  A CTA that covers a whole
// i-block writes the result; the i-blocks cut by a slice boundary get per-CTA
// partial sums that a small fixup kernel adds in CTA order (deterministic, no
// atomics).
//
// Inside a CTA.  Each thread holds IP packed pairs of i-bodies in registers:
// pair q holds bodies 2q*T + t and (2q+1)*T + t of the i-block.  j-tiles
// stream global -> shared through a two-stage ring of 1-D bulk copies (TMA)
// completing on mbarriers; the single issuing thread refills a stage after the
// CTA barrier that ends its use.  Each j-body is one broadcast 32-byte shared
// load of (x,x,y,y,z,z,m,m), then per i-pair 13 packed f32x2 instructions and
// two MUFU reciprocal square roots: the same operation sequence Listing 4
// performs per pair (difference, FMA chain seeded with eps^2, rsqrt cubed,
// times m_j, FMA accumulation, and r2*w for the potential).
//
// Accumulation.  Per tile the sums are plain FP32; with compensation on, each
// tile's partial is folded into a running sum by Kahan summation (four packed
// adds per component per tile, amortised over J pairs), so the per-body sum
// over n terms keeps FP32 pair errors instead of an O(sqrt(n)) FP32 running-sum
// error.  The per-CTA partial sums of split i-blocks are double-float records
// (hi + lo in FP32, the Kahan pair's s - c exactly), added by their consumer
// with FP32 two-sums: no FP64 instruction, which runs at 1/64 of the FP32
// rate on GB300, is left in the epilogue of the mixed kernels.
//
// Self term.  The diagonal tiles (j-tile inside the thread's own i-block) run
// a masked variant that zeroes the pair whose j equals i, so j = i is excluded
// exactly (Eq. 1) and eps = 0 is valid for distinct positions.  Without the
// potential and with eps > 0 the mask is not needed (the pair's difference
// vector is exactly zero) and every tile takes the unmasked loop.
#include <algorithm>
#include <map>
#include <mutex>

#include "nbody_internal.cuh"

namespace nbk {
namespace {

struct KParams {
    const float* jdup;      // sources (packed j-array)
    const double* centres;  // source cell centres (mixed) or nullptr
    const float* ipack;     // sinks: == jdup when the sinks are the sources
    const double* icentres; // sink cell centres (mixed)
    int self;               // sinks are the sources: mask j == i in diagonal tiles
    const int* perm;        // sink slot g holds body perm[g] (nullptr: slot g is body g)
    float eps2;
    int64_t n;              // sinks
    int64_t nblk;
    int64_t gpb;    // granules per i-block row (npad / kGranule)
    int64_t units;  // granules in all: nblk * gpb
    int64_t nctas;
    float* acc;
    float* pot;
    double* partial;  // [nctas][2][block] partial records (four double-float components)
    int* err;
    const int* uni;   // nonzero word: every source has one mass (or nullptr)
};

// One j-tile against the thread's IP i-pairs.
// Kahan step of one packed term into (sum, comp).
__device__ __forceinline__ void kahan_add(f2& sum, f2& comp, f2 term) {
    const f2 y = sub2(term, comp);
    const f2 t = add2(sum, y);
    comp = sub2(sub2(t, sum), y);
    sum = t;
}

// Summation modes: 0 one FP32 running sum, 1 FP32 per tile folded by Kahan
// summation, 2 Kahan summation of every pair term.
// UNI: every source has the same mass; the pair weight leaves m_j out (11
// instead of 12 FP32 operations per interaction) and the caller scales the
// sums by that mass.
// FULL: the whole tile (compile-time bounds); else j-bodies [jlo, jhi) of it
// (multiples of the granule).
template <int T, int IP, int J, int UNROLL, bool POT, bool DIAG, int MODE, int WF, bool UNI, bool FULL>
__device__ __forceinline__ void tile_pass(const unsigned char* tile, const f2 (&xi)[IP], const f2 (&yi)[IP],
                                          const f2 (&zi)[IP], f2 eps2, f2 (&ax)[IP], f2 (&ay)[IP], f2 (&az)[IP],
                                          f2 (&ap)[IP], f2 (&kx)[IP], f2 (&ky)[IP], f2 (&kz)[IP], f2 (&kp)[IP],
                                          int jl0, int tid, int jlo, int jhi) {
    const ulonglong2* tj = reinterpret_cast<const ulonglong2*>(tile);
    const int lo = FULL ? 0 : jlo;
    const int hi = FULL ? J : jhi;
#pragma unroll UNROLL
    for (int j = lo; j < hi; ++j) {
        const ulonglong2 A = tj[2 * j];
        const ulonglong2 B = tj[2 * j + 1];
        const f2 xj = A.x, yj = A.y, zj = B.x, mj = B.y;
#pragma unroll
        for (int q = 0; q < IP; ++q) {
            const f2 dx = sub2(xj, xi[q]);
            const f2 dy = sub2(yj, yi[q]);
            const f2 dz = sub2(zj, zi[q]);
            f2 r2 = fma2(dx, dx, eps2);
            r2 = fma2(dy, dy, r2);
            r2 = fma2(dz, dz, r2);
            float s0, s1;
            upk(r2, s0, s1);
            float q0 = rsqrt_approx(s0);
            float q1 = rsqrt_approx(s1);
            if (DIAG) {
                const int jl = jl0 + j;
                if (jl == 2 * q * T + tid) q0 = 0.0f;
                if (jl == (2 * q + 1) * T + tid) q1 = 0.0f;
            }
            const f2 ri = pk(q0, q1);
            // m_j rsqrt(s)^3 in one of two association orders (the same
            // three products; which schedules better depends on the shape)
            f2 w;
            if (UNI) {
                w = WF == 1 ? mul2(mul2(ri, ri), ri) : mul2(ri, mul2(ri, ri));
            } else if (WF == 1) {
                w = mul2(mul2(ri, ri), mul2(ri, mj));
            } else if (WF == 2) {
                w = mul2(mul2(mul2(ri, mj), ri), ri);
            } else {
                w = mul2(ri, mul2(ri, ri));
                w = mul2(w, mj);
            }
            if (MODE == 2) {
                kahan_add(ax[q], kx[q], mul2(dx, w));
                kahan_add(ay[q], ky[q], mul2(dy, w));
                kahan_add(az[q], kz[q], mul2(dz, w));
                if (POT) kahan_add(ap[q], kp[q], mul2(r2, w));
            } else {
                ax[q] = fma2(dx, w, ax[q]);
                ay[q] = fma2(dy, w, ay[q]);
                az[q] = fma2(dz, w, az[q]);
                if (POT) ap[q] = fma2(r2, w, ap[q]);  // r2 * m_j / r^3 = m_j / r
            }
        }
    }
}

__device__ __forceinline__ void kahan2(f2& sum, f2& comp, f2& part) {
    const f2 y = sub2(part, comp);
    const f2 t = add2(sum, y);
    comp = sub2(sub2(t, sum), y);
    sum = t;
    part = 0ull;
}

// The kernel body.  UNIMODE picks the pair loop: 0 the general loop, 1 the
// equal-mass loop (every source has one mass: m_j left out of the loop, the
// sums scaled by it at the end), 2 either, chosen per j-tile from the flag.
template <int T, int IP, int J, int UNROLL, bool POT, bool MIXED, int KAHAN, int WF, int UNIMODE>
__device__ __forceinline__ void force_body(const KParams& p) {
    constexpr int C = 2 * IP * T;
    constexpr uint32_t TILE_BYTES = J * 32u;
    static_assert(C % J == 0, "a j-tile must not straddle two cells");
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ float s_dc[3];  // MIXED: c_J - c_I of the current j-cell

    const int tid = threadIdx.x;
    const int64_t cta = blockIdx.x;
    constexpr int64_t GPT = J / kGranule;  // granules per j-tile
    static_assert(J % kGranule == 0, "a j-tile is a whole number of granules");
    const int64_t u_begin = cta * p.units / p.nctas;  // this CTA's granules [u_begin, u_end)
    const int64_t u_end = (cta + 1) * p.units / p.nctas;
    // end of the segment (the part of one j-tile inside the slice) starting at granule g
    auto seg_end = [&](int64_t g) { return min(u_end, (g / GPT + 1) * GPT); };
    unsigned char* tiles = smem;
    f2* xsave = reinterpret_cast<f2*>(smem + 2 * TILE_BYTES);  // MIXED: [IP][3][T]

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // the j-tile of the segment starting at granule g (the whole tile is copied)
    auto issue = [&](int s, int64_t g) {
        int64_t tile = (g % p.gpb) / GPT;
        if (!in_range(tile, p.gpb / GPT, p.err)) tile = 0;
        mbar_expect_tx(&bar[s], TILE_BYTES);
        bulk_g2s(tiles + s * TILE_BYTES, p.jdup + tile * (int64_t)J * kJdupFloats, TILE_BYTES, &bar[s]);
    };
    int64_t g_issued = u_begin;  // start of the last segment issued (thread 0's view)
    int in_flight = 0;           // segments issued and not yet consumed (thread 0's view)
    if (tid == 0 && u_begin < u_end) {
        issue(0, u_begin);
        in_flight = 1;
        if (seg_end(u_begin) < u_end) {
            g_issued = seg_end(u_begin);
            issue(1, g_issued);
            in_flight = 2;
        }
    }

    const f2 eps2 = pk(p.eps2, p.eps2);
    // j-slot 0 is always a real body: its mass is every source's mass.
    const bool uni = UNIMODE == 2 ? (p.uni != nullptr && *p.uni != 0) : UNIMODE == 1;
    const float mu = uni ? ld_chain(p.jdup + 6) : 1.0f;
    uint32_t parity = 0;
    int s = 0;
    int64_t u = u_begin;
    bool failed = false;

    while (u < u_end) {
        const int64_t b = u / p.gpb;
        const int64_t ub0 = u;                              // this CTA's first granule of block b
        const int64_t ub1 = min(u_end, (b + 1) * p.gpb);  // and its end
        const int64_t base = b * C;

        f2 xi[IP], yi[IP], zi[IP];
#pragma unroll
        for (int q = 0; q < IP; ++q) {
            int64_t s0 = base + (2 * q) * T + tid, s1 = s0 + T;
            if (!in_range(s0, p.nblk * C, p.err)) s0 = 0;
            if (!in_range(s1, p.nblk * C, p.err)) s1 = 0;
            const float* a0 = p.ipack + s0 * kJdupFloats;
            const float* a1 = p.ipack + s1 * kJdupFloats;
            xi[q] = pk(ld_chain(a0 + 0), ld_chain(a1 + 0));
            yi[q] = pk(ld_chain(a0 + 2), ld_chain(a1 + 2));
            zi[q] = pk(ld_chain(a0 + 4), ld_chain(a1 + 4));
            if (MIXED) {
                xsave[(q * 3 + 0) * T + tid] = xi[q];
                xsave[(q * 3 + 1) * T + tid] = yi[q];
                xsave[(q * 3 + 2) * T + tid] = zi[q];
            }
        }
        f2 ax[IP], ay[IP], az[IP], ap[IP];
        f2 sx[IP], sy[IP], sz[IP], sp[IP], cx[IP], cy[IP], cz[IP], cp[IP];
#pragma unroll
        for (int q = 0; q < IP; ++q) {
            ax[q] = ay[q] = az[q] = ap[q] = 0ull;
            sx[q] = sy[q] = sz[q] = sp[q] = 0ull;
            cx[q] = cy[q] = cz[q] = cp[q] = 0ull;
        }
        int64_t cur_cell = p.self ? b : -1;  // i-offsets start relative to cell b's own centre

        while (u < ub1) {
            const int64_t ue = seg_end(u);  // tiles never straddle i-block rows (gpb is a multiple of GPT)
            const int64_t tt = (u % p.gpb) / GPT;
            const int jlo = (int)(u % GPT) * kGranule, jhi = jlo + (int)(ue - u) * kGranule;
            const bool whole = jlo == 0 && jhi == J;
            const int64_t cell = (tt * J) / C;
            const bool recentre = MIXED && cell != cur_cell;
            if (recentre && tid == 0) {
                // i-coordinates relative to the j-cell's centre: x_i - c_J =
                // (x_i - c_I) - (c_J - c_I), the centre difference in FP64,
                // once per CTA (FP64 is slow on this GPU), shared by the
                // barrier below.
                const double* cj = p.centres + 3 * cell;
                const double* ci = p.icentres + 3 * b;
                s_dc[0] = (float)(ld_chain(cj + 0) - ld_chain(ci + 0));
                s_dc[1] = (float)(ld_chain(cj + 1) - ld_chain(ci + 1));
                s_dc[2] = (float)(ld_chain(cj + 2) - ld_chain(ci + 2));
            }
            const bool ok = mbar_wait_bounded(&bar[s], (parity >> s) & 1u, kWaitLimitNs);
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            parity ^= (1u << s);
            if (recentre) {
                cur_cell = cell;
                const float dx = s_dc[0], dy = s_dc[1], dz = s_dc[2];
                const f2 dx2 = pk(dx, dx), dy2 = pk(dy, dy), dz2 = pk(dz, dz);
#pragma unroll
                for (int q = 0; q < IP; ++q) {
                    xi[q] = sub2(xsave[(q * 3 + 0) * T + tid], dx2);
                    yi[q] = sub2(xsave[(q * 3 + 1) * T + tid], dy2);
                    zi[q] = sub2(xsave[(q * 3 + 2) * T + tid], dz2);
                }
            }
            const unsigned char* tile = tiles + s * TILE_BYTES;
            // The self pair needs the mask only for the potential (it would
            // add m_i/eps) or eps == 0 (0 * inf); otherwise its difference
            // vector is exactly zero (both sides are the same packed entry
            // relative to the same centre) and it adds exactly 0.
            const bool diag = p.self && cell == b && (POT || p.eps2 == 0.0f);
            const bool unil = UNIMODE == 1 || (UNIMODE == 2 && uni);
            const int jl0 = diag ? (int)(tt * J - base) : 0;
#define NBK_TILE(DG, UN, FL)                                                                                       \
    tile_pass<T, IP, J, UNROLL, POT, DG, KAHAN, WF, UN, FL>(tile, xi, yi, zi, eps2, ax, ay, az, ap, cx, cy, cz, cp, \
                                                            jl0, tid, jlo, jhi)
            if (whole) {
                if (diag) {
                    if (unil) NBK_TILE(true, true, true); else NBK_TILE(true, false, true);
                } else {
                    if (unil) NBK_TILE(false, true, true); else NBK_TILE(false, false, true);
                }
            } else {
                if (diag) {
                    if (unil) NBK_TILE(true, true, false); else NBK_TILE(true, false, false);
                } else {
                    if (unil) NBK_TILE(false, true, false); else NBK_TILE(false, false, false);
                }
            }
#undef NBK_TILE
            if (KAHAN == 1) {
#pragma unroll
                for (int q = 0; q < IP; ++q) {
                    kahan2(sx[q], cx[q], ax[q]);
                    kahan2(sy[q], cy[q], ay[q]);
                    kahan2(sz[q], cz[q], az[q]);
                    if (POT) kahan2(sp[q], cp[q], ap[q]);
                }
            }
            __syncthreads();  // every thread is done with stage s
            if (tid == 0) {
                --in_flight;
                const int64_t gn = seg_end(g_issued);  // the segment after the last one issued
                if (gn < u_end) {
                    g_issued = gn;
                    issue(s, gn);
                    ++in_flight;
                }
            }
            s ^= 1;
            u = ue;
        }
        if (failed) break;

        // ---- results of i-block b from this CTA's slice ----
        const bool full = (ub0 == b * p.gpb && ub1 == (b + 1) * p.gpb);
        const int slot = (b == u_begin / p.gpb) ? 0 : 1;
#pragma unroll
        for (int q = 0; q < IP; ++q) {
            // the sums in double-float: a Kahan pair (s, c) is s - c exactly
            DF d[2][4];
            if (MIXED) {
                if (KAHAN != 0) {
                    // mode 1 keeps (sum, comp) in s*, c*; mode 2 in a*, c*
                    const f2 S[4] = {KAHAN == 1 ? sx[q] : ax[q], KAHAN == 1 ? sy[q] : ay[q],
                                     KAHAN == 1 ? sz[q] : az[q], KAHAN == 1 ? sp[q] : ap[q]};
                    const f2 Cm[4] = {cx[q], cy[q], cz[q], cp[q]};
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        float s0, s1, c0, c1;
                        upk(S[k], s0, s1);
                        upk(Cm[k], c0, c1);
                        d[0][k] = two_sum(s0, -c0);
                        d[1][k] = two_sum(s1, -c1);
                    }
                } else {
                    const f2 A[4] = {ax[q], ay[q], az[q], ap[q]};
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        float a0, a1;
                        upk(A[k], a0, a1);
                        d[0][k] = DF{a0, 0.0f};
                        d[1][k] = DF{a1, 0.0f};
                    }
                }
                if (uni) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        d[0][k] = df_scale(d[0][k], mu);
                        d[1][k] = df_scale(d[1][k], mu);
                    }
                }
            } else {
                // The plain kernels keep their FP64 arithmetic here (the sums
                // rounded into double-float at the end): on GB300 the
                // double-float form above scheduled the FP32-state pair loop
                // 3.4 % slower (N = 65536), this one 0.8 %, while the mixed
                // kernels gained 6 % at N = 16384 from dropping the FP64 work.
                double e[2][4];
                if (KAHAN != 0) {
                    const f2 S[4] = {KAHAN == 1 ? sx[q] : ax[q], KAHAN == 1 ? sy[q] : ay[q],
                                     KAHAN == 1 ? sz[q] : az[q], KAHAN == 1 ? sp[q] : ap[q]};
                    const f2 Cm[4] = {cx[q], cy[q], cz[q], cp[q]};
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        float s0, s1, c0, c1;
                        upk(S[k], s0, s1);
                        upk(Cm[k], c0, c1);
                        e[0][k] = (double)s0 - (double)c0;
                        e[1][k] = (double)s1 - (double)c1;
                    }
                } else {
                    float a0, a1;
                    upk(ax[q], a0, a1); e[0][0] = a0; e[1][0] = a1;
                    upk(ay[q], a0, a1); e[0][1] = a0; e[1][1] = a1;
                    upk(az[q], a0, a1); e[0][2] = a0; e[1][2] = a1;
                    upk(ap[q], a0, a1); e[0][3] = a0; e[1][3] = a1;
                }
                if (uni) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        e[0][k] *= (double)mu;
                        e[1][k] *= (double)mu;
                    }
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float h0 = (float)e[0][k], h1 = (float)e[1][k];
                    d[0][k] = DF{h0, (float)(e[0][k] - (double)h0)};
                    d[1][k] = DF{h1, (float)(e[1][k] - (double)h1)};
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int lb = (2 * q + h) * T + tid;
                const int64_t g = base + lb;
                if (full) {
                    if (g < p.n) {
                        const int64_t o = p.perm != nullptr ? (int64_t)p.perm[g] : g;
                        if (!in_range(o, p.n, p.err)) continue;
                        p.acc[3 * o + 0] = df_float(d[h][0]);
                        p.acc[3 * o + 1] = df_float(d[h][1]);
                        p.acc[3 * o + 2] = df_float(d[h][2]);
                        if (POT) p.pot[o] = -df_float(d[h][3]);
                    }
                } else {
                    const int64_t pi = (cta * 2 + slot) * C + lb;
                    if (!in_range(pi, p.nctas * 2 * C, p.err)) continue;
                    store_partial(p.partial, pi, d[h][0], d[h][1], d[h][2], d[h][3]);
                }
            }
        }
    }

    if (failed) {
        if (tid == 0) {
            atomicExch(p.err, kErrTimeout);
            // Let copies still in flight land before shared memory goes away.
            for (int k = 0; k < in_flight; ++k) {
                const int st = (s + k) & 1;
                (void)mbar_wait_bounded(&bar[st], (parity >> st) & 1u, kWaitLimitNs / 4);
            }
        }
        __syncthreads();
    }
}

// The equal-mass choice is made per j-tile in the mixed-precision kernels and
// once per launch (two copies of the body) in the plain ones: on GB300 each
// arrangement scheduled better for its own kernels (measured at N = 2^20,
// log-uniform masses: mixed 71.5 vs 70.7 % of FP32 peak, plain 69.2 vs
// 68.1 %).
template <int T, int IP, int J, int UNROLL, int MINB, bool POT, bool MIXED, int KAHAN, int WF>
__global__ void __launch_bounds__(T, MINB) force_kernel(const KParams p) {
    pdl_trigger();
    pdl_wait();  // the packed j-array of this evaluation is complete
    if (MIXED)
        force_body<T, IP, J, UNROLL, POT, MIXED, KAHAN, WF, 2>(p);
    else if (p.uni != nullptr && *p.uni != 0)
        force_body<T, IP, J, UNROLL, POT, MIXED, KAHAN, WF, 1>(p);
    else
        force_body<T, IP, J, UNROLL, POT, MIXED, KAHAN, WF, 0>(p);
}

// Adds the per-CTA partial sums of every i-block that a slice boundary cut,
// in CTA order.  Grid (i-block, chunk of blockDim.x bodies of the block), so
// a few large blocks still spread over many SMs; blocks covered by one CTA
// return at once.
__global__ void fixup_kernel(const KParams p, int C, int pot_on) {
    pdl_trigger();
    pdl_wait();  // every CTA of the force kernel has written its partial sums
    const int64_t b = blockIdx.x;
    int64_t c_lo, c_hi;
    int slot_lo;
    split_ctas(b, p.gpb, p.units, p.nctas, &c_lo, &c_hi, &slot_lo);
    if (c_lo == c_hi) return;
    for (int lb = blockIdx.y * blockDim.x + threadIdx.x; lb < C; lb += gridDim.y * blockDim.x) {
        const int64_t g = b * C + lb;
        if (g >= p.n) break;
        if (!in_range((c_hi * 2) * C + lb, p.nctas * 2 * C, p.err)) continue;
        float s4[4];
        split_sum(p.partial, C, b, c_lo, c_hi, slot_lo, lb, s4);
        const int64_t o = p.perm != nullptr ? (int64_t)p.perm[g] : g;
        if (!in_range(o, p.n, p.err)) continue;
        p.acc[3 * o + 0] = s4[0];
        p.acc[3 * o + 1] = s4[1];
        p.acc[3 * o + 2] = s4[2];
        if (pot_on) p.pot[o] = -s4[3];
    }
}

typedef void (*KernelFn)(const KParams);

struct ShapeEntry {
    ForceShape shape;  // shape.jtile: the mixed-precision kernels' j-tile
    int jt[2];         // j-tile of the [plain, mixed] kernels
    int cap;  // most CTAs per SM the persistent grid uses (16 warps per SM)
    KernelFn fn[2][2][3];  // [pot][mixed][summation mode]
    size_t smem(bool mixed) const {
        return 2u * jt[mixed ? 1 : 0] * 32u + (mixed ? (size_t)shape.ipairs * 3 * shape.threads * 8 : 0);
    }
};

// WF0: association order of m_j rsqrt(s)^3 in the kernels without the
// potential (those with it use order 0).  J, UNROLL: j-tile and j-unroll of
// the mixed-precision kernels; JP, UP: of the plain ones (the best pair
// differs between the two on some shapes).
template <int T, int IP, int J, int UNROLL, int MINB, int WF0 = 0, int JP = J, int UP = UNROLL>
ShapeEntry make_entry() {
    ShapeEntry e;
    e.shape = ForceShape{T, IP, J, 2 * IP * T};
    e.jt[0] = JP;
    e.jt[1] = J;
    e.cap = T >= 512 ? 1 : 512 / T;
    e.fn[0][0][0] = force_kernel<T, IP, JP, UP, MINB, false, false, 0, WF0>;
    e.fn[0][0][1] = force_kernel<T, IP, JP, UP, MINB, false, false, 1, WF0>;
    e.fn[0][0][2] = force_kernel<T, IP, JP, UP, MINB, false, false, 2, WF0>;
    e.fn[0][1][0] = force_kernel<T, IP, J, UNROLL, MINB, false, true, 0, WF0>;
    e.fn[0][1][1] = force_kernel<T, IP, J, UNROLL, MINB, false, true, 1, WF0>;
    e.fn[0][1][2] = force_kernel<T, IP, J, UNROLL, MINB, false, true, 2, WF0>;
    e.fn[1][0][0] = force_kernel<T, IP, JP, UP, MINB, true, false, 0, 0>;
    e.fn[1][0][1] = force_kernel<T, IP, JP, UP, MINB, true, false, 1, 0>;
    e.fn[1][0][2] = force_kernel<T, IP, JP, UP, MINB, true, false, 2, 0>;
    e.fn[1][1][0] = force_kernel<T, IP, J, UNROLL, MINB, true, true, 0, 0>;
    e.fn[1][1][1] = force_kernel<T, IP, J, UNROLL, MINB, true, true, 1, 0>;
    e.fn[1][1][2] = force_kernel<T, IP, J, UNROLL, MINB, true, true, 2, 0>;
    return e;
}

const ShapeEntry* shapes() {
    static const ShapeEntry table[] = {
        make_entry<256, 4, 256, 4, 0>(),  // 0: 2048-body blocks (fastest with the potential)
        make_entry<256, 2, 256, 4, 0>(),  // 1: 1024
        make_entry<512, 2, 1024, 2, 0, 1, 512, 4>(),  // 2: 2048 (fastest without the potential)
        make_entry<128, 2, 128, 2, 0>(),  // 3: 512
        make_entry<128, 1, 64, 2, 0>(),   // 4: 256 (small n)
#ifdef NBODY_EXTRA_SHAPES
        make_entry<256, 2, 256, 2, 0>(),  // 5
        make_entry<256, 2, 256, 2, 3>(),  // 6
        make_entry<256, 2, 256, 1, 0>(),  // 7
        make_entry<512, 2, 256, 2, 0>(),  // 8
        make_entry<128, 2, 256, 2, 0>(),  // 9
        make_entry<256, 3, 256, 2, 0>(),  // 10
        make_entry<384, 2, 256, 2, 0>(),  // 11
        make_entry<256, 2, 512, 2, 0>(),  // 12
        make_entry<256, 1, 256, 4, 0>(),  // 13
        make_entry<256, 2, 128, 2, 0>(),  // 14
        make_entry<256, 2, 256, 2, 2>(),  // 15
        make_entry<256, 2, 256, 8, 0>(),  // 16
        make_entry<512, 2, 256, 4, 0>(),  // 17
        make_entry<256, 2, 512, 4, 0>(),  // 18
        make_entry<256, 4, 256, 4, 0>(),  // 19
        make_entry<256, 2, 256, 4, 2>(),  // 20
        make_entry<128, 2, 128, 4, 0>(),  // 21
        make_entry<128, 1, 64, 4, 0>(),   // 22
        make_entry<64, 2, 128, 4, 0>(),   // 23
        make_entry<512, 2, 256, 2, 0, 1>(),   // 24
        make_entry<512, 2, 256, 8, 0, 1>(),   // 25
        make_entry<512, 2, 128, 4, 0, 1>(),   // 26
        make_entry<512, 2, 256, 4, 0, 1>(),   // 27
        make_entry<1024, 1, 256, 4, 0, 1>(),  // 28
        make_entry<512, 1, 256, 4, 0, 1>(),   // 29
        make_entry<512, 3, 256, 4, 0, 1>(),   // 30
        make_entry<256, 2, 256, 4, 0, 2>(),   // 31
        make_entry<512, 2, 256, 4, 0, 2>(),   // 32
        make_entry<384, 2, 256, 4, 0, 1>(),   // 33
        make_entry<128, 2, 256, 4, 0, 1>(),   // 34
        make_entry<256, 2, 512, 4, 0, 1>(),   // 35
        make_entry<512, 4, 256, 4, 0, 1>(),   // 36
        make_entry<512, 2, 512, 4, 0, 1>(),   // 37 (shape 2 before 1024-body j-tiles)
#endif
    };
    return table;
}
#ifdef NBODY_EXTRA_SHAPES
constexpr int kNumShapes = 38;
#else
constexpr int kNumShapes = 5;
#endif

// Resident CTAs per SM for each kernel variant, queried once per device (the
// dynamic shared-memory limit each variant needs is a per-device attribute,
// set on the device that is current at the first launch there).
struct OccTable {
    int v[kNumShapes][2][2][3];
    OccTable() {
        for (int a = 0; a < kNumShapes; ++a)
            for (int b = 0; b < 2; ++b)
                for (int c = 0; c < 2; ++c)
                    for (int d = 0; d < 3; ++d) v[a][b][c][d] = -1;
    }
};
std::mutex g_occ_mu;
std::map<int, OccTable> g_occ;

int occupancy(int k, int pot, int mixed, int kahan) {
    int dev = 0;
    (void)cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_occ_mu);
    int& o = g_occ[dev].v[k][pot][mixed][kahan];
    if (o < 0) {
        const ShapeEntry& e = shapes()[k];
        const size_t sm = e.smem(mixed);
        cudaFuncSetAttribute(e.fn[pot][mixed][kahan], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, e.fn[pot][mixed][kahan], e.shape.threads, sm) !=
                cudaSuccess ||
            nb < 1)
            nb = 1;
        o = nb;
    }
    return o;
}

}  // namespace

int force_num_shapes() { return kNumShapes; }
ForceShape force_shape(int k) { return shapes()[k].shape; }

size_t force_partial_doubles(int k, int num_sms) {
    // Upper bound over variants: at most 4 resident CTAs of any shape fit the
    // register file at the shapes compiled here; 8 leaves margin.
    const ForceShape s = shapes()[k].shape;
    return (size_t)num_sms * 8u * 2u * (size_t)s.block * 4u;
}

cudaError_t split_fixup(int64_t n, int64_t nblk, int64_t gpb, int64_t nctas, int block, const double* partial,
                        float* out3, float* out1, cudaStream_t st, const int* perm, int* err) {
    KParams p;
    p.jdup = nullptr;
    p.centres = nullptr;
    p.ipack = nullptr;
    p.icentres = nullptr;
    p.self = 1;
    p.perm = perm;
    p.eps2 = 0.0f;
    p.n = n;
    p.nblk = nblk;
    p.gpb = gpb;
    p.units = nblk * gpb;
    p.nctas = nctas;
    p.acc = out3;
    p.pot = out1;
    p.partial = const_cast<double*>(partial);
    p.err = err;
    p.uni = nullptr;
    return launch_pdl(fixup_kernel, dim3((unsigned)nblk, (unsigned)((block + 255) / 256)), dim3(256), 0, st, p, block,
                      out1 != nullptr ? 1 : 0);
}

size_t force_partial_doubles_for(int k, bool pot, bool mixed, bool compensated, int64_t npad, int num_sms) {
    const ShapeEntry& e = shapes()[k];
    const int occ = std::min(occupancy(k, pot ? 1 : 0, mixed ? 1 : 0, compensated ? 1 : 0), e.cap);  // mode 0 or 1
    const int64_t units = (npad / e.shape.block) * (npad / kGranule);
    const int64_t nctas = std::min<int64_t>((int64_t)num_sms * occ, units);
    return (size_t)nctas * 2u * (size_t)e.shape.block * 4u;
}

cudaError_t force_launch(int k, const ForceArgs& a, int num_sms, cudaStream_t st, int* launched, cudaEvent_t ev0,
                         cudaEvent_t ev1, SplitSums* defer) {
    const ShapeEntry& e = shapes()[k];
    const int C = e.shape.block;
    const int pot = a.pot != nullptr, mixed = a.centres != nullptr, kahan = a.summation;
    KParams p;
    p.jdup = a.jdup;
    p.centres = a.centres;
    p.ipack = a.ipack != nullptr ? a.ipack : a.jdup;
    p.icentres = a.ipack != nullptr ? a.icentres : a.centres;
    p.self = a.ipack == nullptr ? 1 : 0;
    p.perm = a.perm;
    p.eps2 = a.eps2;
    p.n = a.n;
    p.nblk = (a.ipack != nullptr ? a.nipad : a.npad) / C;
    p.gpb = a.npad / kGranule;
    p.units = p.nblk * p.gpb;
    int occ = occupancy(k, pot, mixed, kahan);
    occ = std::min(occ, e.cap);
    p.nctas = std::min<int64_t>((int64_t)num_sms * occ, p.units);
    p.acc = a.acc;
    p.pot = a.pot;
    p.partial = a.partial;
    p.err = a.err;
    p.uni = a.uni;
    const size_t sm = e.smem(mixed);
    *launched = 0;
    if (ev0 != nullptr) cudaEventRecord(ev0, st);
    cudaError_t err = launch_pdl(e.fn[pot][mixed][kahan], dim3((unsigned)p.nctas), dim3(e.shape.threads), sm, st, p);
    if (err != cudaSuccess) return err;
    *launched = 1;
    if (ev1 != nullptr) cudaEventRecord(ev1, st);
    if (defer != nullptr) {  // the pack kernel that consumes these accelerations adds the partials
        defer->partial = p.nctas > 1 ? p.partial : nullptr;
        defer->units = p.units;
        defer->nctas = p.nctas;
        defer->gpb = p.gpb;
        defer->block = C;
        return cudaSuccess;
    }
    if (p.nctas > 1) {  // a single CTA covers every i-block whole
        err = launch_pdl(fixup_kernel, dim3((unsigned)p.nblk, (unsigned)((C + 255) / 256)), dim3(256), 0, st, p, C,
                         pot);
        if (err == cudaSuccess) *launched = 2;
    }
    return err;
}

}  // namespace nbk
