// vjp.cu -- reverse mode of the all-pairs force (Eq. 1 of Miki & Hanawa,
// Sec. III.A): the vector-Jacobian product through the tidal tensor, as a
// second all-pairs pass, plus the O(n) kernels of the leapfrog's adjoint sweep.
//
// For cotangents lam_i of the accelerations (and optionally mu_i of the
// potentials), with d = r_j - r_k, s = |d|^2 + eps^2 and
// T(d) = s^{-3/2} I - 3 s^{-5/2} d d^T:
//   dL/dr_k = sum_{j != k} T(d) u_kj,   u_kj = m_k lam_j - m_j lam_k
//             - sum_j s^{-3/2} d (mu_j m_k + mu_k m_j)               (potential)
//   dL/dm_k = -sum_{j != k} [ s^{-3/2} (lam_j . d) + mu_j s^{-1/2} ]
// (body k is the source of every pair (i, k) and the sink of every pair
// (k, j); T(d) = T(-d) lets both be gathered at k).  Per pair that is 29
// packed FP32 operations and two MUFU reciprocal square roots, against 12 for
// the force.
//
// The kernel mirrors the force kernel: stream-K persistent grid over
// (i-block, 32 j-body granule) units, i-bodies packed in f32x2 pairs in registers, j-tiles
// of 64 bytes per body (x, y, z, m, lam, mu, each duplicated) staged by 1-D
// bulk copies on a two-stage mbarrier ring with bounded waits, masked diagonal
// tiles for j = k, FP64 cell centres for mixed precision, and per-tile FP32
// partials folded into FP32 totals (two-level summation).
#include <algorithm>
#include <map>
#include <mutex>
#include <type_traits>

#include "nbody_internal.cuh"

namespace nbk {
namespace {

constexpr int kVjpFloats = 16;  // x x y y z z m m lx lx ly ly lz lz mu mu

struct VParams {
    const float* jv;
    const double* centres;
    float eps2;
    int64_t n;
    int64_t nblk;
    int64_t gpb;    // granules per i-block row (npad / kGranule)
    int64_t units;  // granules in all: nblk * gpb
    int64_t nctas;
    float* g_pos;
    float* g_mass;
    float* acc;           // FORCE kernels: the force at the same positions, [n][3]
    double* partial;      // [nctas][2][block] partial records: (g_pos, -g_mass) of split blocks
    double* partial_acc;  // FORCE kernels: [nctas][2][block] partial records (acc, 0), after the VJP's
    int* err;
    const int* uni;  // nonzero word: every body has one mass (or nullptr)
};

// UNI: every body has the same mass mu; u = m_k lam_j - m_j lam_k becomes
// mu (lam_j - lam_k), formed without the masses (26 instead of 29 packed
// operations per pair), and the caller scales the position gradient by mu.
// FULL: the whole tile; else j-bodies [jlo, jhi) of it (granule multiples).
// FORCE: also the force a_k = sum_j m_j s^{-3/2} d at the same positions (3
// more FMAs per pair; 4 with distinct masses), into (fx, fy, fz).
template <int T, int IP, int J, int UNROLL, bool MU, bool DIAG, bool UNI, bool FULL, bool FORCE>
__device__ __forceinline__ void vjp_tile(const unsigned char* tile, const f2 (&xi)[IP], const f2 (&yi)[IP],
                                         const f2 (&zi)[IP], const f2 (&nlx)[IP], const f2 (&nly)[IP],
                                         const f2 (&nlz)[IP], const f2 (&mi)[IP], const f2 (&nmi)[IP],
                                         const f2 (&nmui)[IP], f2 eps2,
                                         f2 (&gx)[IP], f2 (&gy)[IP], f2 (&gz)[IP], f2 (&gm)[IP], f2 (&fx)[IP],
                                         f2 (&fy)[IP], f2 (&fz)[IP], int jl0, int tid, int jlo, int jhi) {
    const ulonglong2* tj = reinterpret_cast<const ulonglong2*>(tile);
    const f2 m3 = pk(-3.0f, -3.0f);
    const int lo = FULL ? 0 : jlo;
    const int hi = FULL ? J : jhi;
#pragma unroll UNROLL
    for (int j = lo; j < hi; ++j) {
        const ulonglong2 A = tj[4 * j + 0];
        const ulonglong2 B = tj[4 * j + 1];
        const ulonglong2 Cc = tj[4 * j + 2];
        const ulonglong2 D = tj[4 * j + 3];
        const f2 xj = A.x, yj = A.y, zj = B.x, mj = B.y, lxj = Cc.x, lyj = Cc.y, lzj = D.x, muj = D.y;
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
            const f2 ri2 = mul2(ri, ri);
            const f2 r3 = mul2(ri, ri2);
            // u = m_k lam_j - m_j lam_k (UNI: lam_j - lam_k, times mu later)
            const f2 ux = UNI ? add2(lxj, nlx[q]) : fma2(mi[q], lxj, mul2(mj, nlx[q]));
            const f2 uy = UNI ? add2(lyj, nly[q]) : fma2(mi[q], lyj, mul2(mj, nly[q]));
            const f2 uz = UNI ? add2(lzj, nlz[q]) : fma2(mi[q], lzj, mul2(mj, nlz[q]));
            f2 du = mul2(dx, ux);
            du = fma2(dy, uy, du);
            du = fma2(dz, uz, du);
            // T(d) u = s^{-3/2} (u - 3 s^{-1} (d.u) d): the same two terms as
            // s^{-3/2} u - 3 s^{-5/2} (d.u) d, one product fewer per pair
            const f2 e = mul2(mul2(ri2, m3), du);  // -3 s^{-1} (d.u)
            gx[q] = fma2(r3, fma2(e, dx, ux), gx[q]);
            gy[q] = fma2(r3, fma2(e, dy, uy), gy[q]);
            gz[q] = fma2(r3, fma2(e, dz, uz), gz[q]);
            f2 dl = mul2(dx, lxj);
            dl = fma2(dy, lyj, dl);
            dl = fma2(dz, lzj, dl);
            gm[q] = fma2(r3, dl, gm[q]);
            if (FORCE) {
                const f2 w = UNI ? r3 : mul2(r3, mj);
                fx[q] = fma2(dx, w, fx[q]);
                fy[q] = fma2(dy, w, fy[q]);
                fz[q] = fma2(dz, w, fz[q]);
            }
            if (MU) {
                // -s^{-3/2} d (mu_j m_k + mu_k m_j) with d = r_j - r_k, and mu_j s^{-1/2};
                // nmi, nmui hold -m_k, -mu_k
                const f2 cm = UNI ? mul2(r3, sub2(nmui[q], muj)) : mul2(r3, fma2(muj, nmi[q], mul2(nmui[q], mj)));
                gx[q] = fma2(cm, dx, gx[q]);
                gy[q] = fma2(cm, dy, gy[q]);
                gz[q] = fma2(cm, dz, gz[q]);
                gm[q] = fma2(muj, ri, gm[q]);
            }
        }
    }
}

template <int T, int IP, int J, int UNROLL, bool MU, bool MIXED, bool FORCE>
__global__ void __launch_bounds__(T) vjp_kernel(const VParams p) {
    pdl_trigger();
    pdl_wait();  // the packed j-array of this step is complete
    constexpr int C = 2 * IP * T;
    constexpr uint32_t TILE_BYTES = J * kVjpFloats * 4u;
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
    auto seg_end = [&](int64_t g) { return min(u_end, (g / GPT + 1) * GPT); };
    unsigned char* tiles = smem;
    f2* xsave = reinterpret_cast<f2*>(smem + 2 * TILE_BYTES);  // MIXED: [IP][3][T]

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int s, int64_t g) {
        int64_t tile = (g % p.gpb) / GPT;
        if (!in_range(tile, p.gpb / GPT, p.err)) tile = 0;
        mbar_expect_tx(&bar[s], TILE_BYTES);
        bulk_g2s(tiles + s * TILE_BYTES, p.jv + tile * (int64_t)J * kVjpFloats, TILE_BYTES, &bar[s]);
    };
    int64_t g_issued = u_begin;
    int in_flight = 0;
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
    // One mass for every body (j-slot 0 is always a real body): the pair loop
    // leaves the masses out of u and the position gradient is scaled by mu.
    const bool uni = p.uni != nullptr && *p.uni != 0;
    const float mu = uni ? ld_chain(p.jv + 6) : 1.0f;
    uint32_t parity = 0;
    int s = 0;
    int64_t u = u_begin;
    bool failed = false;

    while (u < u_end) {
        const int64_t b = u / p.gpb;
        const int64_t ub0 = u;
        const int64_t ub1 = min(u_end, (b + 1) * p.gpb);
        const int64_t base = b * C;
        f2 xi[IP], yi[IP], zi[IP], nlx[IP], nly[IP], nlz[IP], mi[IP], nmi[IP], nmui[IP];
#pragma unroll
        for (int q = 0; q < IP; ++q) {
            int64_t s0 = base + (2 * q) * T + tid, s1 = s0 + T;
            if (!in_range(s0, p.nblk * C, p.err)) s0 = 0;
            if (!in_range(s1, p.nblk * C, p.err)) s1 = 0;
            const float* a0 = p.jv + s0 * kVjpFloats;
            const float* a1 = p.jv + s1 * kVjpFloats;
            xi[q] = pk(ld_chain(a0 + 0), ld_chain(a1 + 0));
            yi[q] = pk(ld_chain(a0 + 2), ld_chain(a1 + 2));
            zi[q] = pk(ld_chain(a0 + 4), ld_chain(a1 + 4));
            mi[q] = pk(ld_chain(a0 + 6), ld_chain(a1 + 6));
            nlx[q] = pk(-ld_chain(a0 + 8), -ld_chain(a1 + 8));
            nly[q] = pk(-ld_chain(a0 + 10), -ld_chain(a1 + 10));
            nlz[q] = pk(-ld_chain(a0 + 12), -ld_chain(a1 + 12));
            nmi[q] = pk(-ld_chain(a0 + 6), -ld_chain(a1 + 6));
            nmui[q] = pk(-ld_chain(a0 + 14), -ld_chain(a1 + 14));
            if (MIXED) {
                xsave[(q * 3 + 0) * T + tid] = xi[q];
                xsave[(q * 3 + 1) * T + tid] = yi[q];
                xsave[(q * 3 + 2) * T + tid] = zi[q];
            }
        }
        f2 gx[IP], gy[IP], gz[IP], gm[IP], tx[IP], ty[IP], tz[IP], tm[IP];
        f2 fx[IP], fy[IP], fz[IP], ux[IP], uy[IP], uz[IP];  // FORCE: per tile, and totals
#pragma unroll
        for (int q = 0; q < IP; ++q) {
            gx[q] = gy[q] = gz[q] = gm[q] = tx[q] = ty[q] = tz[q] = tm[q] = 0ull;
            fx[q] = fy[q] = fz[q] = ux[q] = uy[q] = uz[q] = 0ull;
        }
        int64_t cur_cell = b;

        while (u < ub1) {
            const int64_t ue = seg_end(u);
            const int64_t tt = (u % p.gpb) / GPT;
            const int jlo = (int)(u % GPT) * kGranule, jhi = jlo + (int)(ue - u) * kGranule;
            const bool whole = jlo == 0 && jhi == J;
            const int64_t cell = (tt * J) / C;
            const bool recentre = MIXED && cell != cur_cell;
            if (recentre && tid == 0) {  // c_J - c_I in FP64 once per CTA, shared by the barrier below
                const double* cj = p.centres + 3 * cell;
                const double* ci = p.centres + 3 * b;
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
                const float ddx = s_dc[0], ddy = s_dc[1], ddz = s_dc[2];
                const f2 dx2 = pk(ddx, ddx), dy2 = pk(ddy, ddy), dz2 = pk(ddz, ddz);
#pragma unroll
                for (int q = 0; q < IP; ++q) {
                    xi[q] = sub2(xsave[(q * 3 + 0) * T + tid], dx2);
                    yi[q] = sub2(xsave[(q * 3 + 1) * T + tid], dy2);
                    zi[q] = sub2(xsave[(q * 3 + 2) * T + tid], dz2);
                }
            }
            const unsigned char* tile = tiles + s * TILE_BYTES;
            // With one mass for all bodies, no potential cotangent and eps > 0
            // the self pair adds exactly 0 (u = mu (lam_k - lam_k) = 0 and the
            // difference vector is zero), so only the other cases mask it.
            const bool diag = cell == b && (MU || !uni || p.eps2 == 0.0f);
            const int jl0 = diag ? (int)(tt * J - base) : 0;
#define NBK_VTILE(DG, UN, FL)                                                                                 \
    vjp_tile<T, IP, J, UNROLL, MU, DG, UN, FL, FORCE>(tile, xi, yi, zi, nlx, nly, nlz, mi, nmi, nmui, eps2, gx, gy, gz, \
                                                      gm, fx, fy, fz, jl0, tid, jlo, jhi)
            if (whole) {
                if (diag) {
                    if (uni) NBK_VTILE(true, true, true); else NBK_VTILE(true, false, true);
                } else {
                    if (uni) NBK_VTILE(false, true, true); else NBK_VTILE(false, false, true);
                }
            } else {
                if (diag) {
                    if (uni) NBK_VTILE(true, true, false); else NBK_VTILE(true, false, false);
                } else {
                    if (uni) NBK_VTILE(false, true, false); else NBK_VTILE(false, false, false);
                }
            }
#undef NBK_VTILE
#pragma unroll
            for (int q = 0; q < IP; ++q) {
                tx[q] = add2(tx[q], gx[q]);
                ty[q] = add2(ty[q], gy[q]);
                tz[q] = add2(tz[q], gz[q]);
                tm[q] = add2(tm[q], gm[q]);
                gx[q] = gy[q] = gz[q] = gm[q] = 0ull;
                if (FORCE) {
                    ux[q] = add2(ux[q], fx[q]);
                    uy[q] = add2(uy[q], fy[q]);
                    uz[q] = add2(uz[q], fz[q]);
                    fx[q] = fy[q] = fz[q] = 0ull;
                }
            }
            __syncthreads();
            if (tid == 0) {
                --in_flight;
                const int64_t gn = seg_end(g_issued);
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

        const bool full = (ub0 == b * p.gpb && ub1 == (b + 1) * p.gpb);
        const int slot = (b == u_begin / p.gpb) ? 0 : 1;
#pragma unroll
        for (int q = 0; q < IP; ++q) {
            float v[2][4], f[2][3];
            upk(tx[q], v[0][0], v[1][0]);
            upk(ty[q], v[0][1], v[1][1]);
            upk(tz[q], v[0][2], v[1][2]);
            upk(tm[q], v[0][3], v[1][3]);
            if (FORCE) {
                upk(ux[q], f[0][0], f[1][0]);
                upk(uy[q], f[0][1], f[1][1]);
                upk(uz[q], f[0][2], f[1][2]);
            }
            if (uni) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    v[0][k] *= mu;
                    v[1][k] *= mu;
                    if (FORCE) {
                        f[0][k] *= mu;
                        f[1][k] *= mu;
                    }
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int lb = (2 * q + h) * T + tid;
                const int64_t g = base + lb;
                if (full) {
                    if (g < p.n) {
                        if (!in_range(g, p.n, p.err)) continue;
                        p.g_pos[3 * g + 0] = v[h][0];
                        p.g_pos[3 * g + 1] = v[h][1];
                        p.g_pos[3 * g + 2] = v[h][2];
                        p.g_mass[g] = -v[h][3];
                        if (FORCE) {
                            p.acc[3 * g + 0] = f[h][0];
                            p.acc[3 * g + 1] = f[h][1];
                            p.acc[3 * g + 2] = f[h][2];
                        }
                    }
                } else {
                    const int64_t pi = (cta * 2 + slot) * C + lb;
                    if (!in_range(pi, p.nctas * 2 * C, p.err)) continue;
                    store_partial(p.partial, pi, DF{v[h][0], 0.0f}, DF{v[h][1], 0.0f}, DF{v[h][2], 0.0f},
                                  DF{v[h][3], 0.0f});
                    if (FORCE)
                        store_partial(p.partial_acc, pi, DF{f[h][0], 0.0f}, DF{f[h][1], 0.0f}, DF{f[h][2], 0.0f},
                                      DF{0.0f, 0.0f});
                }
            }
        }
    }

    if (failed) {
        if (tid == 0) {
            atomicExch(p.err, kErrTimeout);
            for (int k = 0; k < in_flight; ++k) {
                const int st = (s + k) & 1;
                (void)mbar_wait_bounded(&bar[st], (parity >> st) & 1u, kWaitLimitNs / 4);
            }
        }
        __syncthreads();
    }
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

__device__ __forceinline__ void store_jv(float* jv, int64_t k, float x, float y, float z, float m, float lx, float ly,
                                         float lz, float mu) {
    float4* d = reinterpret_cast<float4*>(jv + k * kVjpFloats);
    d[0] = make_float4(x, x, y, y);
    d[1] = make_float4(z, z, m, m);
    d[2] = make_float4(lx, lx, ly, ly);
    d[3] = make_float4(lz, lz, mu, mu);
}

// The VJP's j-array, built as the force's FP64 pack is: two body-parallel
// kernels over 256-slot chunks.  The first does the adjoint-sweep updates
// (when lamx != nullptr)
//   lamx += g_prev, gm_acc += gm_prev, lam += drift * lamx
// (g_prev and gm_prev from the previous VJP, or from its deferred partial sums)
// and each chunk's FP64 position sum; the second the cell centres (mixed) and
// the entries with cotangent kappa * lam, relative to the centre (mixed) or
// absolute (plain).
constexpr int kVChunk = 256;

// FUSED (mixed precision, every pack of the adjoint sweep after its first):
// the same kernel also writes the j-array entries, relative to each cell's
// centre taken one step earlier -- the mean of the cell's positions from the
// chunk sums the previous pack left in fz.chunks_in -- so the sweep step is
// one kernel instead of two; its own chunk sums go to `chunks` for the next.
constexpr int kVMaxChunksPerCell = 8;  // blocks of up to 2048 bodies
struct VjpFused {
    int block = 0;
    const double* chunks_in = nullptr;
    const float* mass = nullptr;
    double kappa = 0.0;
    float* jv = nullptr;
    double* centres = nullptr;
};

template <typename L, bool FUSED = false>
__global__ void __launch_bounds__(kVChunk, 1) vjp_step_kernel(int64_t n, const double* __restrict__ pos,
                                                           L* __restrict__ lam, double* __restrict__ lamx,
                                                           const float* __restrict__ gprev,
                                                           const float* __restrict__ gmprev,
                                                           double* __restrict__ gm_acc, double drift,
                                                           double* __restrict__ chunks, const SplitSums ss,
                                                           const ReverseStep rev, const VjpFused fz) {
    pdl_trigger();
    __shared__ double red[3][kVChunk / 32];
    __shared__ float redf[3][kVChunk / 32];
    __shared__ double cin[3 * kVMaxChunksPerCell];
    __shared__ double cen[3];
    const int tid = threadIdx.x;
    const int64_t g = (int64_t)blockIdx.x * kVChunk + tid;
    // Before the wait: arithmetic on the launch parameters, and (FUSED) the
    // masses, which no kernel of the sweep writes.
    const BlockSplit bs = block_split(ss, (int64_t)blockIdx.x * kVChunk);
    const BlockSplit ba = block_split(rev.ss_acc, (int64_t)blockIdx.x * kVChunk);
    const int per_cell = FUSED ? fz.block / kVChunk : 1;
    const int64_t cell = (int64_t)blockIdx.x / per_cell;
    float mg = 0.0f;
    if (FUSED && g < n) mg = fz.mass[g];
    pdl_wait();  // the previous VJP (and force) results are complete
    // FUSED: the cell's chunk sums of one step earlier, for its centre
    if (FUSED && tid < 3 * per_cell) cin[tid] = ld_chain(fz.chunks_in + 3 * cell * per_cell + tid);
    double lv[3] = {0.0, 0.0, 0.0};  // FUSED: the updated cotangent lam of this body
    double x = 0.0, y = 0.0, z = 0.0;
    double r[3] = {0.0, 0.0, 0.0};  // positions after the reverse step (pos aliases rev.x then)
    if (g < n && rev.x != nullptr) {  // the leapfrog step s run backwards
        double w[3];
        if (rev.anchor_x != nullptr) {
            for (int c = 0; c < 3; ++c) {
                r[c] = rev.anchor_x[3 * g + c];
                w[c] = rev.anchor_v[3 * g + c];
            }
        } else {
            float a3[3] = {0.0f, 0.0f, 0.0f};
            if (rev.a != nullptr) split_acc<16>(rev.ss_acc, ba, g, g, rev.a, a3);
            for (int c = 0; c < 3; ++c) {
                w[c] = ld_chain(rev.vh + 3 * g + c) - rev.kick * (double)a3[c];
                r[c] = ld_chain(rev.x + 3 * g + c) - rev.drift * w[c];
            }
        }
        for (int c = 0; c < 3; ++c) {
            rev.x[3 * g + c] = r[c];
            rev.vh[3 * g + c] = w[c];
        }
    }
    if (g < n) {
        if constexpr (!std::is_const<L>::value) {
            if (lamx != nullptr) {
                float gp[3] = {0.0f, 0.0f, 0.0f};
                float gmp = 0.0f;
                if (gprev != nullptr) {
                    bool split = false;
                    if (ss.partial != nullptr) {  // the previous VJP's partials, summed as its fixup would
                        if (bs.c_lo < bs.c_hi) {
                            float s4[4];
                            split_sum<16>(ss.partial, ss.block, bs.b, bs.c_lo, bs.c_hi, bs.slot_lo,
                                          (int)(g - bs.b * ss.block), s4);
                            gp[0] = s4[0];
                            gp[1] = s4[1];
                            gp[2] = s4[2];
                            gmp = -s4[3];
                            split = true;
                        }
                    }
                    if (!split) {
                        gp[0] = ld_chain(gprev + 3 * g + 0);
                        gp[1] = ld_chain(gprev + 3 * g + 1);
                        gp[2] = ld_chain(gprev + 3 * g + 2);
                        gmp = gmprev != nullptr ? ld_chain(gmprev + g) : 0.0f;
                    }
                }
                for (int c = 0; c < 3; ++c) {
                    double lx = ld_chain(lamx + 3 * g + c);
                    if (gprev != nullptr) lx += (double)gp[c];
                    lamx[3 * g + c] = lx;
                    lv[c] = (double)(L)((double)ld_chain(lam + 3 * g + c) + drift * lx);
                    lam[3 * g + c] = (L)lv[c];
                }
                if (gmprev != nullptr) gm_acc[g] = ld_chain(gm_acc + g) + (double)gmp;
            }
        }
        if (rev.x != nullptr) {
            x = r[0];
            y = r[1];
            z = r[2];
        } else {
            x = ld_chain(pos + 3 * g + 0);
            y = ld_chain(pos + 3 * g + 1);
            z = ld_chain(pos + 3 * g + 2);
        }
    }
    if (FUSED) {
        __syncthreads();  // the chunk sums are in shared memory
        if (tid < 3) {  // as vjp_offsets_kernel computes it (the same sums in the same order)
            double t = 0.0;
            for (int q = 0; q < per_cell; ++q) t += cin[3 * q + tid];
            const int64_t base = cell * fz.block;
            const int64_t cnt = (n - base) < fz.block ? (n - base) : (int64_t)fz.block;
            cen[tid] = t / (double)cnt;
            if (blockIdx.x % per_cell == 0) fz.centres[3 * cell + tid] = cen[tid];
        }
        __syncthreads();
        float ox = 0.0f, oy = 0.0f, oz = 0.0f;
        if (g < n) {
            ox = (float)(x - cen[0]);
            oy = (float)(y - cen[1]);
            oz = (float)(z - cen[2]);
            store_jv(fz.jv, g, ox, oy, oz, mg, (float)(fz.kappa * lv[0]), (float)(fz.kappa * lv[1]),
                     (float)(fz.kappa * lv[2]), 0.0f);
        } else {
            store_jv(fz.jv, g, kPadPos, kPadPos, kPadPos, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f);
        }
        // the chunk's position sum for the next step's centres: its body count
        // times this centre plus the FP32 sum of its offsets (any point near
        // the cell serves as a centre; no FP64 reduction)
        ox = warp_sum_f(ox);
        oy = warp_sum_f(oy);
        oz = warp_sum_f(oz);
        if ((tid & 31) == 0) {
            redf[0][tid >> 5] = ox;
            redf[1][tid >> 5] = oy;
            redf[2][tid >> 5] = oz;
        }
        __syncthreads();
        if (tid < 3) {
            float t = 0.0f;
            for (int q = 0; q < kVChunk / 32; ++q) t += redf[tid][q];
            const int64_t left = n - (int64_t)blockIdx.x * kVChunk;
            const int64_t cnt = left < 0 ? 0 : (left < kVChunk ? left : (int64_t)kVChunk);
            chunks[3 * (int64_t)blockIdx.x + tid] = (double)cnt * cen[tid] + (double)t;
        }
        return;
    }
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
        for (int q = 0; q < kVChunk / 32; ++q) t += red[tid][q];
        chunks[3 * (int64_t)blockIdx.x + tid] = t;
    }
}

template <typename L>
__global__ void __launch_bounds__(kVChunk) vjp_offsets_kernel(int64_t n, int block, const double* __restrict__ pos,
                                                              const float* __restrict__ mass,
                                                              const L* __restrict__ lam, double kappa,
                                                              const float* __restrict__ mu, int plain,
                                                              float* __restrict__ jv, double* __restrict__ centres,
                                                              const double* __restrict__ chunks) {
    pdl_trigger();
    pdl_wait();  // every chunk's positions, adjoints and sums are written
    __shared__ double cen[3];
    const int tid = threadIdx.x;
    const int64_t ch = blockIdx.x;
    const int per_cell = block / kVChunk;
    const int64_t cell = ch / per_cell;
    if (tid < 3) {
        double c = 0.0;
        if (!plain) {
            double t = 0.0;
            for (int q = 0; q < per_cell; ++q) t += ld_chain(chunks + 3 * (cell * per_cell + q) + tid);
            const int64_t base = cell * block;
            const int64_t cnt = (n - base) < block ? (n - base) : (int64_t)block;
            c = t / (double)cnt;
            if (ch % per_cell == 0) centres[3 * cell + tid] = c;
        }
        cen[tid] = c;
    }
    __syncthreads();
    const int64_t g = ch * kVChunk + tid;
    if (g < n) {
        store_jv(jv, g, (float)(ld_chain(pos + 3 * g + 0) - cen[0]), (float)(ld_chain(pos + 3 * g + 1) - cen[1]),
                 (float)(ld_chain(pos + 3 * g + 2) - cen[2]), mass[g],
                 (float)(kappa * (double)ld_chain(lam + 3 * g + 0)), (float)(kappa * (double)ld_chain(lam + 3 * g + 1)),
                 (float)(kappa * (double)ld_chain(lam + 3 * g + 2)), mu ? mu[g] : 0.0f);
    } else {
        store_jv(jv, g, kPadPos, kPadPos, kPadPos, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f);
    }
}

// lamx += g, gm_acc += gm (the last step of the adjoint sweep).
__global__ void adjoint_accumulate_kernel(int64_t n, double* __restrict__ lamx, const float* __restrict__ g,
                                          double* __restrict__ gm_acc, const float* __restrict__ gm) {
    pdl_trigger();
    pdl_wait();  // the last VJP's results are complete
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < 3 * n; k += (int64_t)gridDim.x * blockDim.x) {
        lamx[k] = ld_chain(lamx + k) + (double)ld_chain(g + k);
        if (k < n) gm_acc[k] = ld_chain(gm_acc + k) + (double)ld_chain(gm + k);
    }
}

typedef void (*VFn)(const VParams);
struct VShapeEntry {
    VjpShape shape;
    VFn fn[2][2];  // [mu][mixed]
    VFn fnf[2];    // [mixed]: with the force, no potential cotangent
    size_t smem(bool mixed) const {
        return 2u * shape.jtile * kVjpFloats * 4u + (mixed ? (size_t)shape.ipairs * 3 * shape.threads * 8 : 0);
    }
};

template <int T, int IP, int J, int UNROLL>
VShapeEntry make_ventry() {
    VShapeEntry e;
    e.shape = VjpShape{T, IP, J, 2 * IP * T};
    e.fn[0][0] = vjp_kernel<T, IP, J, UNROLL, false, false, false>;
    e.fn[0][1] = vjp_kernel<T, IP, J, UNROLL, false, true, false>;
    e.fn[1][0] = vjp_kernel<T, IP, J, UNROLL, true, false, false>;
    e.fn[1][1] = vjp_kernel<T, IP, J, UNROLL, true, true, false>;
    e.fnf[0] = vjp_kernel<T, IP, J, UNROLL, false, false, true>;
    e.fnf[1] = vjp_kernel<T, IP, J, UNROLL, false, true, true>;
    return e;
}

const VShapeEntry* vshapes() {
    static const VShapeEntry table[] = {
        make_ventry<256, 2, 128, 2>(),  // 0: 1024-body blocks
        make_ventry<128, 2, 128, 2>(),  // 1: 512
        make_ventry<256, 1, 128, 4>(),  // 2: 512
        make_ventry<128, 1, 64, 2>(),   // 3: 256
    };
    return table;
}
constexpr int kNumVShapes = 4;

// Resident CTAs per SM for each variant, queried once per device (the
// shared-memory attribute is set per device).
struct VOccTable {
    int v[kNumVShapes][3][2];  // [shape][0: VJP, 1: with mu, 2: with the force][mixed]
    VOccTable() {
        for (int a = 0; a < kNumVShapes; ++a)
            for (int b = 0; b < 3; ++b)
                for (int c = 0; c < 2; ++c) v[a][b][c] = -1;
    }
};
std::mutex g_vocc_mu;
std::map<int, VOccTable> g_vocc;

int vocc(int k, int mu, int mixed) {
    int dev = 0;
    (void)cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_vocc_mu);
    int& o = g_vocc[dev].v[k][mu][mixed];
    if (o < 0) {
        const VShapeEntry& e = vshapes()[k];
        const size_t sm = e.smem(mixed);
        VFn fn = mu == 2 ? e.fnf[mixed] : e.fn[mu][mixed];
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, e.shape.threads, sm) != cudaSuccess ||
            nb < 1)
            nb = 1;
        o = std::min(nb, 8);
    }
    return o;
}

}  // namespace

int vjp_num_shapes() { return kNumVShapes; }
VjpShape vjp_shape(int k) { return vshapes()[k].shape; }
int vjp_floats_per_body() { return kVjpFloats; }

// Two halves: the VJP's partials, then (FORCE launches) the force's.
size_t vjp_partial_doubles(int k, int num_sms) {
    return 2 * (size_t)num_sms * 8u * 2u * (size_t)vshapes()[k].shape.block * 4u;
}

cudaError_t pack_vjp(int64_t n, int64_t npad, int block, const double* pos, const float* mass, const float* lam_f32,
                     double* lam_f64, double* lamx, const float* gprev, const float* gmprev, double* gm_acc,
                     double drift, double kappa, const float* mu, bool plain, float* jv, double* centres,
                     cudaStream_t st, const SplitSums* ss, const ReverseStep* rev) {
    if (block % kVChunk != 0 || npad % block != 0) return cudaErrorInvalidValue;
    const unsigned nch = (unsigned)(npad / kVChunk);
    double* chunks = centres + 3 * (npad / block);
    const SplitSums sv = ss != nullptr ? *ss : SplitSums();
    const ReverseStep rv = rev != nullptr ? *rev : ReverseStep();
    if (rev != nullptr && rev->x != nullptr) pos = rev->x;
    if (lam_f64 != nullptr) {
        cudaError_t e = launch_pdl(vjp_step_kernel<double>, dim3(nch), dim3(kVChunk), 0, st, n, pos, lam_f64, lamx, gprev,
                                   gmprev, gm_acc, drift, chunks, sv, rv, VjpFused());
        if (e != cudaSuccess) return e;
        return launch_pdl(vjp_offsets_kernel<double>, dim3(nch), dim3(kVChunk), 0, st, n, block, pos, mass,
                          (const double*)lam_f64, kappa, mu, plain ? 1 : 0, jv, centres, (const double*)chunks);
    }
    cudaError_t e = launch_pdl(vjp_step_kernel<const float>, dim3(nch), dim3(kVChunk), 0, st, n, pos, lam_f32,
                               (double*)nullptr, (const float*)nullptr, (const float*)nullptr, (double*)nullptr, 0.0,
                               chunks, sv, rv, VjpFused());
    if (e != cudaSuccess) return e;
    return launch_pdl(vjp_offsets_kernel<const float>, dim3(nch), dim3(kVChunk), 0, st, n, block, pos, mass, lam_f32,
                      kappa, mu, plain ? 1 : 0, jv, centres, (const double*)chunks);
}

cudaError_t pack_vjp_lagged(int64_t n, int64_t npad, int block, const float* mass, double* lam_f64, double* lamx,
                            const float* gprev, const float* gmprev, double* gm_acc, double drift, double kappa,
                            float* jv, double* centres, const double* chunks_in, double* chunks_out,
                            cudaStream_t st, const SplitSums* ss, const ReverseStep* rev) {
    if (block % kVChunk != 0 || block / kVChunk > kVMaxChunksPerCell || npad % block != 0 || lam_f64 == nullptr ||
        lamx == nullptr || rev == nullptr || rev->x == nullptr)
        return cudaErrorInvalidValue;
    VjpFused fz;
    fz.block = block;
    fz.chunks_in = chunks_in;
    fz.mass = mass;
    fz.kappa = kappa;
    fz.jv = jv;
    fz.centres = centres;
    return launch_pdl(vjp_step_kernel<double, true>, dim3((unsigned)(npad / kVChunk)), dim3(kVChunk), 0, st, n,
                      (const double*)rev->x, lam_f64, lamx, gprev, gmprev, gm_acc, drift, chunks_out,
                      ss != nullptr ? *ss : SplitSums(), *rev, fz);
}

cudaError_t adjoint_accumulate(int64_t n, double* lamx, const float* g, double* gm_acc, const float* gm,
                               cudaStream_t st) {
    int64_t grid = (3 * n + 255) / 256;
    const int64_t cap = (int64_t)current_sms() * 16;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    return launch_pdl(adjoint_accumulate_kernel, dim3((unsigned)grid), dim3(256), 0, st, n, lamx, g, gm_acc, gm);
}

cudaError_t vjp_launch(int k, const VjpArgs& a, int num_sms, cudaStream_t st, int* launched, cudaEvent_t ev0,
                       cudaEvent_t ev1, SplitSums* defer, SplitSums* defer_acc) {
    const VShapeEntry& e = vshapes()[k];
    const int C = e.shape.block;
    const int mu = a.has_mu ? 1 : 0, mixed = a.centres != nullptr ? 1 : 0;
    const bool force = a.acc != nullptr && !a.has_mu;
    VParams p;
    p.jv = a.jv;
    p.centres = a.centres;
    p.eps2 = a.eps2;
    p.n = a.n;
    p.nblk = a.npad / C;
    p.gpb = a.npad / kGranule;
    p.units = p.nblk * p.gpb;
    p.nctas = std::min<int64_t>((int64_t)num_sms * vocc(k, force ? 2 : mu, mixed), p.units);
    p.g_pos = a.g_pos;
    p.g_mass = a.g_mass;
    p.acc = force ? a.acc : nullptr;
    p.partial = a.partial;
    p.partial_acc = a.partial + (size_t)p.nctas * 2 * C * 4;
    p.err = a.err;
    p.uni = a.uni;
    *launched = 0;
    if (ev0 != nullptr) cudaEventRecord(ev0, st);
    VFn fn = force ? e.fnf[mixed] : e.fn[mu][mixed];
    cudaError_t err = launch_pdl(fn, dim3((unsigned)p.nctas), dim3(e.shape.threads), e.smem(mixed), st, p);
    if (err != cudaSuccess) return err;
    *launched = 1;
    if (ev1 != nullptr) cudaEventRecord(ev1, st);
    auto describe = [&](SplitSums* d, double* part) {
        d->partial = p.nctas > 1 ? part : nullptr;
        d->units = p.units;
        d->nctas = p.nctas;
        d->gpb = p.gpb;
        d->block = C;
    };
    if (force && defer_acc != nullptr) {
        describe(defer_acc, p.partial_acc);
    } else if (force && p.nctas > 1) {
        err = split_fixup(p.n, p.nblk, p.gpb, p.nctas, C, p.partial_acc, p.acc, nullptr, st, nullptr, p.err);
        if (err != cudaSuccess) return err;
        *launched += 1;
    }
    if (defer != nullptr) {  // the next pack_vjp adds the split blocks' partials
        describe(defer, p.partial);
        return cudaSuccess;
    }
    if (p.nctas > 1) {
        err = split_fixup(p.n, p.nblk, p.gpb, p.nctas, C, p.partial, p.g_pos, p.g_mass, st, nullptr, p.err);
        if (err == cudaSuccess) *launched += 1;
    }
    return err;
}

}  // namespace nbk
