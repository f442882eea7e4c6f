// k_fluid.cu -- lattice kernels of the coupled LB-MD step:
//   * the fused pull-scheme stream + bounce-back + moments + BGK collide
//     (Sec. II, Eqs. 1-5, with the walls of Sec. III), with the per-step
//     mass/momentum diagnostics folded in as exact fixed-point sums;
//   * the sparse source pass that adds the beads' reaction (Sec. II, Eq. 9) at
//     the lattice sites the beads touched;
//   * state transfer (equilibrium initialisation, pull to / push from the
//     fp32 staging area) and the fluid part of the observables.
#include "lbmd_internal.cuh"

#include <utility>

namespace lbmd {

// ---------------------------------------------------------------------------
// Fluid diagnostics sums.  Each block turns its threads' FP32 partials of
// rho - 1 and rho u into 64-bit fixed point (fix_of), sums them exactly and
// adds them to its realization's accumulator with four integer atomics: no
// fence, no completion counter, and a result independent of order and of the
// launch shape.  A later kernel in stream order reads the accumulator,
// converts it to FP64 and zeroes it (the source kernel for the per-step row,
// the bead observables kernel for the observables).  FP64 arithmetic, slow
// on this GPU, is left to those few conversions.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void block_partial4(float a, float b, float c, float d, long long *acc, int *status) {
    __shared__ long long s[16][4];
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = tid & 31, warp = tid >> 5, nw = (blockDim.x * blockDim.y + 31) >> 5;
    if (!(isfinite(a) && isfinite(b) && isfinite(c) && isfinite(d))) atomicOr(status, ST_NONFINITE);
    const long long v0 = warp_sum_ll(fix_of(a, FIXD_FLUID)), v1 = warp_sum_ll(fix_of(b, FIXD_FLUID));
    const long long v2 = warp_sum_ll(fix_of(c, FIXD_FLUID)), v3 = warp_sum_ll(fix_of(d, FIXD_FLUID));
    if (lane == 0) { s[warp][0] = v0; s[warp][1] = v1; s[warp][2] = v2; s[warp][3] = v3; }
    __syncthreads();
    if (tid < 4) {
        long long t = 0;
        for (int w = 0; w < nw; ++w) t += s[w][tid];
        if (t != 0) atomicAdd(reinterpret_cast<unsigned long long *>(acc) + tid, (unsigned long long)t);
    }
}

// c_i . (x, y, z) for a D3Q19 velocity (components in {-1, 0, 1}): only the
// nonzero components enter, so an axis velocity costs no instruction and an
// edge velocity one addition
template <int I>
__device__ __forceinline__ float cdot(float x, float y, float z) {
    float s = 0.0f;
    bool any = false;
    if (cx(I) != 0) { s = cx(I) > 0 ? x : -x; any = true; }
    if (cy(I) != 0) { const float t = cy(I) > 0 ? y : -y; s = any ? s + t : t; any = true; }
    if (cz(I) != 0) { const float t = cz(I) > 0 ? z : -z; s = any ? s + t : t; }
    return s;
}

// BGK relaxation of one site in stored units (h, or h * 2^12 for FP16).
// With j = rho u the equilibrium (Eq. 5) reads
//   heq_i = w_i [ K + 9/2 (c_i.u)(c_i.j) + 3 c_i.j ],   K = (rho - 1) - 3/2 u.j,
// since rho (c.u) = c.j.  The relaxation (Eq. 4) then is
//   hr_i = (1 - om) h_i + om heq_i,
// and an opposite pair (i, i + 1) (c_{i+1} = -c_i) shares
//   E = om w_i (K + 9/2 (c_i.u)(c_i.j)),   O = 3 om w_i c_i.j:
//   hr_i = (1 - om) h_i + (E + O),   hr_{i+1} = (1 - om) h_{i+1} + (E - O).
// Out: hr, the moment sums in stored units (rho - 1, j) and rho.
template <int PREC>
__device__ __forceinline__ void bgk_relax(const float (&h)[Q], float om, float (&hr)[Q], float &drho_s, float &jx,
                                          float &jy, float &jz, float &rho) {
    constexpr float down = PopScale<PREC>::down;
    // moments from the sums and differences of the opposite pairs
    drho_s = h[0];
    jx = 0.f; jy = 0.f; jz = 0.f;
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const float sp = h[i] + h[i + 1], dp = h[i] - h[i + 1];
        drho_s += sp;
        if (cx(i) == 1) jx += dp;
        if (cx(i) == -1) jx -= dp;
        if (cy(i) == 1) jy += dp;
        if (cy(i) == -1) jy -= dp;
        if (cz(i) == 1) jz += dp;
        if (cz(i) == -1) jz -= dp;
    }
    rho = 1.0f + drho_s * down;
    const float t = (1.5f * down) / rho;  // v = 3/2 u (the scale power of two is exact)
    const float vx = jx * t, vy = jy * t, vz = jz * t;
    const float K = drho_s - (vx * jx + vy * jy + vz * jz);
    const float c1 = 1.0f - om;
    hr[0] = c1 * h[0] + (om * wq(0)) * K;
    // weight classes: axis velocities (wq 1/18), edge velocities (1/36)
    const float oa = om * wq(1), oe = om * wq(7);
    const float ka = oa * K, ke = oe * K;
    const float ax = (3.0f * oa) * jx, ay = (3.0f * oa) * jy, az = (3.0f * oa) * jz;
    const float ex = (3.0f * oe) * jx, ey = (3.0f * oe) * jy, ez = (3.0f * oe) * jz;
#define LBMD_PAIR(I)                                                                                           \
    {                                                                                                          \
        constexpr bool edge = (cx(I) != 0) + (cy(I) != 0) + (cz(I) != 0) == 2;                                 \
        const float O = edge ? cdot<I>(ex, ey, ez) : cdot<I>(ax, ay, az);                                      \
        const float E = fmaf(cdot<I>(vx, vy, vz), O, edge ? ke : ka);                                          \
        hr[I] = fmaf(c1, h[I], E + O);                                                                         \
        hr[I + 1] = fmaf(c1, h[I + 1], E - O);                                                                 \
    }
    LBMD_PAIR(1) LBMD_PAIR(3) LBMD_PAIR(5) LBMD_PAIR(7) LBMD_PAIR(9) LBMD_PAIR(11) LBMD_PAIR(13) LBMD_PAIR(15)
    LBMD_PAIR(17)
#undef LBMD_PAIR
}

// ---------------------------------------------------------------------------
// Fused pull stream + bounce-back + moments + BGK collision.
//   h_i(x)   = h*_i(x - c_i)          pulled from A, or h*_opp(i)(x) when x - c_i is solid
//   rho      = 1 + sum_i h_i,  rho u = sum_i h_i c_i               (Eqs. 1-2)
//   h*_i     = h_i + omega (heq_i - h_i) + 3 w_i g.c_i              (Eqs. 4-5)
//   heq_i    = w_i [ (rho - 1) + rho (3 c.u + 9/2 (c.u)^2 - 3/2 u.u) ]
// (h = f - w; the arithmetic is bgk_relax's).  Block (32, by) covers 32 consecutive x of `by` rows; each thread
// walks zc consecutive z planes.  MODE 0: store; 1: store + per-step sums;
// 2: sums only (observables).
// ---------------------------------------------------------------------------
template <int PREC, int MODE, int U, bool FL>
__global__ void __launch_bounds__(512, FL ? 1 : 2) k_stream_collide(const Sim S, const void *__restrict__ Av,
                                                        void *__restrict__ Bv, const int zc,
                                                        const int nzb) {
    using T = typename PopT<PREC>::T;
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int r = blockIdx.z / nzb;
    const int z0 = (blockIdx.z - r * nzb) * zc;
    const int nx = S.nx, ny = S.ny, nz = S.nz;
    const uint32_t ns = (uint32_t)S.ps;  // population stride (padded site count)
    const T *__restrict__ A = reinterpret_cast<const T *>(Av) + (size_t)r * Q * ns;
    T *__restrict__ B = reinterpret_cast<T *>(Bv) + (size_t)r * Q * ns;
    long long step = 0;
    if (MODE == 1 || FL) step = S.ctrl->step;
    float am = 0.f, ax = 0.f, ay = 0.f, az = 0.f;
    const float om = S.omega;
    const float g0 = S.g[0], g1 = S.g[1], g2 = S.g[2];
    const bool has_g = (g0 != 0.f) || (g1 != 0.f) || (g2 != 0.f);

    if (x < nx && y < ny) {
        const int xv0 = (x == 0 ? nx - 1 : x - 1), xv2 = (x == nx - 1 ? 0 : x + 1);
        const int yv0 = (y == 0 ? ny - 1 : y - 1), yv2 = (y == ny - 1 ? 0 : y + 1);
        const int zend = min(z0 + zc, nz);
        for (int zb = z0; zb < zend; zb += U) {
          // issue the loads of U consecutive sites before any arithmetic, so
          // that 19 * U loads per thread are in flight together
          float hh[U][Q];
          uint32_t lmu[U];
          int su[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int z = zb + u;
            lmu[u] = SOLID_BIT;
            su[u] = 0;
            if (z >= zend) continue;
            const int zv0 = (z == 0 ? nz - 1 : z - 1), zv2 = (z == nz - 1 ? 0 : z + 1);
            const int s = x + nx * (y + ny * z);
            su[u] = s;
            // warp-uniform: a flagged tile holds a bounce-back link somewhere
            if (S.tileflag[blockIdx.x + S.nxt * (y + ny * z)]) {
                const uint32_t lm = __ldg(S.link + s);
                lmu[u] = lm;
                if (lm & SOLID_BIT) continue;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const int sx = cx(i) == 1 ? xv0 : (cx(i) == -1 ? xv2 : x);
                    const int sy = cy(i) == 1 ? yv0 : (cy(i) == -1 ? yv2 : y);
                    const int sz = cz(i) == 1 ? zv0 : (cz(i) == -1 ? zv2 : z);
                    const uint32_t src = (uint32_t)(sx + nx * (sy + ny * sz));
                    const bool bb = (lm >> i) & 1u;
                    const uint32_t idx = bb ? (uint32_t)opp(i) * ns + (uint32_t)s : (uint32_t)i * ns + src;
                    hh[u][i] = load_raw(A, idx);
                }
            } else {  // no bounce-back in the tile: plain pull
                lmu[u] = 0u;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const int sx = cx(i) == 1 ? xv0 : (cx(i) == -1 ? xv2 : x);
                    const int sy = cy(i) == 1 ? yv0 : (cy(i) == -1 ? yv2 : y);
                    const int sz = cz(i) == 1 ? zv0 : (cz(i) == -1 ? zv2 : z);
                    hh[u][i] = load_raw(A, (uint32_t)i * ns + (uint32_t)(sx + nx * (sy + ny * sz)));
                }
            }
          }
          // arithmetic in stored units (h, or h * 2^12 for FP16): the moments
          // are scaled once, so no population is (the scale is a power of two:
          // the results are those of the unscaled formulas)
          constexpr float up = PopScale<PREC>::up, down = PopScale<PREC>::down;
#pragma unroll
          for (int u = 0; u < U; ++u) {
            if (lmu[u] & SOLID_BIT) continue;
            const int s = su[u];
            float hr[Q], drho_s, jx, jy, jz, rho;
            bgk_relax<PREC>(hh[u], om, hr, drho_s, jx, jy, jz, rho);
            if (MODE != 0 && x >= S.own_lo && x < S.own_hi) {
                am += drho_s * down; ax += jx * down; ay += jy * down; az += jz * down;
            }
            if (MODE != 2) {
                // fluctuating LB: mode k (4..18) gets amplitude sqrt(rho) fl_amp[k-4] r_k
                float am_[15];
                if (FL) {
                    float z[16];
                    fluid_noise16(S.seed, S.real_base + (uint32_t)r, (uint32_t)s, step, z);
                    const float sr = sqrtf(fmaxf(rho, 0.0f)) * up;
#pragma unroll
                    for (int k = 0; k < 15; ++k) am_[k] = sr * S.fl_amp[k] * z[k];
                }
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    float hn = hr[i];
                    if (FL) {
                        float d = 0.0f;
#pragma unroll
                        for (int k = 4; k < Q; ++k)
                            if (mode_e(k, i) != 0.0f) d += mode_e(k, i) * am_[k - 4];
                        hn += wq(i) * d;
                    }
                    if (has_g)
                        hn += up * (3.0f * wq(i) * ((float)cx(i) * g0 + (float)cy(i) * g1 + (float)cz(i) * g2));
                    store_raw(B, (uint32_t)i * ns + (uint32_t)s, hn);
                }
            }
          }
        }
    }
    if (MODE != 0)
        block_partial4(am, ax, ay, az, S.fsum + 4 * ((size_t)(MODE == 2 ? S.n_real : 0) + r), &S.ctrl->status);
}

// ---------------------------------------------------------------------------
// The lattice pass with two x sites per thread (x0 = 2k and x0 + 1): a warp
// covers 64 consecutive sites of one row.  Every link's source row is read as
// aligned pairs, one 8-byte (FP32) or 4-byte (FP16) load for both sites; a
// c_x = +-1 link takes the site beyond the pair from the neighbouring lane's
// pair by a shuffle, and the warp's end lanes (or the lane next to the
// periodic wrap) load that one directly.  Stores go as pairs, except in tiles
// with a bounce-back link, which store site by site (solid sites are never
// written, as in k_stream_collide).  Every address and the loop overhead
// serve two sites.  The per-site arithmetic is k_stream_collide's
// (bgk_relax); no thermal noise.  Needs an even nx.  Blocks of
// at most 256 threads, three per SM: 80 registers, no spills (left free, the
// compiler takes 128 and holds half the warps: FP16 135 instead of 107 us).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 pair_load(const float *base, uint32_t idx) {
    return __ldg(reinterpret_cast<const float2 *>(base + idx));
}
__device__ __forceinline__ float2 pair_load(const __half *base, uint32_t idx) {
    return __half22float2(__ldg(reinterpret_cast<const __half2 *>(base + idx)));
}
__device__ __forceinline__ void pair_store(float *base, uint32_t idx, float a, float b) {
    *reinterpret_cast<float2 *>(base + idx) = make_float2(a, b);
}
__device__ __forceinline__ void pair_store(__half *base, uint32_t idx, float a, float b) {
    *reinterpret_cast<__half2 *>(base + idx) = __floats2half2_rn(a, b);
}

// BGK update of one site from its pulled h (stored units): hn, and the
// site's moments (unscaled) for the diagnostics sums
template <int PREC>
__device__ __forceinline__ void bgk_site(const float (&h)[Q], float om, bool has_g, float g0f, float g1f, float g2f,
                                         float (&hn)[Q], float &drho, float &jx, float &jy, float &jz) {
    constexpr float up = PopScale<PREC>::up, down = PopScale<PREC>::down;
    float drho_s, rho;
    bgk_relax<PREC>(h, om, hn, drho_s, jx, jy, jz, rho);
    drho = drho_s * down;
    jx *= down; jy *= down; jz *= down;
    if (has_g) {
#pragma unroll
        for (int i = 0; i < Q; ++i)
            hn[i] += up * (3.0f * wq(i) * ((float)cx(i) * g0f + (float)cy(i) * g1f + (float)cz(i) * g2f));
    }
}

template <int PREC, int MODE>
__global__ void __launch_bounds__(256, 3) k_stream_collide_x2(const Sim S, const void *__restrict__ Av,
                                                              void *__restrict__ Bv, const int zc, const int nzb) {
    using T = typename PopT<PREC>::T;
    const int lane = threadIdx.x;
    const int x0 = 2 * (blockIdx.x * 32 + lane);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int r = blockIdx.z / nzb;
    const int z0 = (blockIdx.z - r * nzb) * zc;
    const int nx = S.nx, ny = S.ny, nz = S.nz;
    const uint32_t ns = (uint32_t)S.ps;
    const T *__restrict__ A = reinterpret_cast<const T *>(Av) + (size_t)r * Q * ns;
    T *__restrict__ B = reinterpret_cast<T *>(Bv) + (size_t)r * Q * ns;
    float am = 0.f, ax = 0.f, ay = 0.f, az = 0.f;
    const float om = S.omega;
    const float g0f = S.g[0], g1f = S.g[1], g2f = S.g[2];
    const bool has_g = (g0f != 0.f) || (g1f != 0.f) || (g2f != 0.f);
    const bool act = x0 < nx;

    if (y < ny) {  // warp-uniform: a warp is one row
        const int xl = x0 == 0 ? nx - 1 : x0 - 1;           // the site before the pair (periodic)
        const int xr = x0 + 2 >= nx ? x0 + 2 - nx : x0 + 2;  // the site after it
        const bool edge_l = lane == 0, edge_r = lane == 31 || x0 + 2 >= nx;
        const int yv0 = (y == 0 ? ny - 1 : y - 1), yv2 = (y == ny - 1 ? 0 : y + 1);
        const int zend = min(z0 + zc, nz);
        for (int z = z0; z < zend; ++z) {
            const int zv0 = (z == 0 ? nz - 1 : z - 1), zv2 = (z == nz - 1 ? 0 : z + 1);
            const int s0 = x0 + nx * (y + ny * z);
            float h0[Q], h1[Q];
            // every lane takes part in the shuffles; lanes past nx load nothing
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int sy = cy(i) == 1 ? yv0 : (cy(i) == -1 ? yv2 : y);
                const int sz = cz(i) == 1 ? zv0 : (cz(i) == -1 ? zv2 : z);
                const uint32_t row = (uint32_t)i * ns + (uint32_t)(nx * (sy + ny * sz));
                float2 c = make_float2(0.f, 0.f);
                if (act) c = pair_load(A, row + (uint32_t)x0);
                if (cx(i) == 0) {
                    h0[i] = c.x;
                    h1[i] = c.y;
                } else if (cx(i) == 1) {  // from x - 1: site x0 - 1 is the previous lane's second
                    float e = __shfl_up_sync(0xffffffffu, c.y, 1);
                    if (act && edge_l) e = load_raw(A, row + (uint32_t)xl);
                    h0[i] = e;
                    h1[i] = c.x;
                } else {  // from x + 1: site x0 + 2 is the next lane's first
                    float e = __shfl_down_sync(0xffffffffu, c.x, 1);
                    if (act && edge_r) e = load_raw(A, row + (uint32_t)xr);
                    h0[i] = c.y;
                    h1[i] = e;
                }
            }
            if (!act) continue;
            // a flagged tile (x0 and x0 + 1 share it) holds a bounce-back link somewhere
            uint32_t lm0 = 0u, lm1 = 0u;
            const bool flagged = S.tileflag[(x0 >> 5) + S.nxt * (y + ny * z)] != 0;
            if (flagged) {
                const uint2 lw = __ldg(reinterpret_cast<const uint2 *>(S.link + s0));
                lm0 = lw.x;
                lm1 = lw.y;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    if ((lm0 >> i) & 1u) h0[i] = load_raw(A, (uint32_t)opp(i) * ns + (uint32_t)s0);
                    if ((lm1 >> i) & 1u) h1[i] = load_raw(A, (uint32_t)opp(i) * ns + (uint32_t)s0 + 1u);
                }
            }
            float n0[Q], n1[Q], d0, jx0, jy0, jz0, d1, jx1, jy1, jz1;
            bgk_site<PREC>(h0, om, has_g, g0f, g1f, g2f, n0, d0, jx0, jy0, jz0);
            bgk_site<PREC>(h1, om, has_g, g0f, g1f, g2f, n1, d1, jx1, jy1, jz1);
            const bool f0 = !(lm0 & SOLID_BIT), f1 = !(lm1 & SOLID_BIT);
            if (MODE != 0) {
                if (f0 && x0 >= S.own_lo && x0 < S.own_hi) { am += d0; ax += jx0; ay += jy0; az += jz0; }
                if (f1 && x0 + 1 >= S.own_lo && x0 + 1 < S.own_hi) { am += d1; ax += jx1; ay += jy1; az += jz1; }
            }
            if (!flagged) {
#pragma unroll
                for (int i = 0; i < Q; ++i) pair_store(B, (uint32_t)i * ns + (uint32_t)s0, n0[i], n1[i]);
            } else {
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    if (f0) store_raw(B, (uint32_t)i * ns + (uint32_t)s0, n0[i]);
                    if (f1) store_raw(B, (uint32_t)i * ns + (uint32_t)s0 + 1u, n1[i]);
                }
            }
        }
    }
    if (MODE != 0) block_partial4(am, ax, ay, az, S.fsum + 4 * (size_t)r, &S.ctrl->status);
}

bool x2_lattice_ok(const Sim &S) { return !S.fluct && S.nx % 2 == 0; }

cudaError_t launch_stream_collide_x2(const Sim &S, const void *A, void *B, int by, int zc, bool diag,
                                     cudaStream_t st) {
    if (!x2_lattice_ok(S) || by < 1 || by > 8 || zc < 1) return cudaErrorInvalidValue;
    const int nzb = (S.nz + zc - 1) / zc;
    const dim3 grid((S.nx + 63) / 64, (S.ny + by - 1) / by, nzb * S.n_real), block(32, by);
#define X2_LAUNCH(P, M) k_stream_collide_x2<P, M><<<grid, block, 0, st>>>(S, A, B, zc, nzb)
    if (S.precision == LBMD_FP16DEV) {
        if (diag) X2_LAUNCH(1, 1); else X2_LAUNCH(1, 0);
    } else {
        if (diag) X2_LAUNCH(0, 1); else X2_LAUNCH(0, 0);
    }
#undef X2_LAUNCH
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The lattice pass fed by tensor copies.  A CTA of 256 threads owns a run of
// row groups; a group is floor(256 / nx) consecutive x rows (rows over y, then
// z, then realizations), one thread per site.  For every row of a group and
// every link i, one cp.async.bulk.tensor copies the source row (y - c_iy,
// z - c_iz), wrapped periodically, into a ring of shared-memory stages that
// an mbarrier per stage tracks; the x shift -c_ix (also periodic) is an index
// into that row.  A stage is refilled once every thread has used it.  Each
// CTA keeps up to STAGES groups in flight, far more bytes than its registers
// could hold, so fewer SMs reach the HBM rate.  Bounce-back links and solid
// sites are read from global memory, as in k_stream_collide, whose per-site
// arithmetic this is.  Waits are bounded: a CTA that gives up latches
// ST_TIMEOUT, waits (bounded) for its copies in flight and leaves.
// ---------------------------------------------------------------------------
constexpr int TMA_THREADS = 256;
template <int PREC> struct TmaStages;
template <> struct TmaStages<0> { static constexpr int n = 4; };  // 4 x 19.5 KB with 256-site rows
template <> struct TmaStages<1> { static constexpr int n = 8; };  // 8 x 9.7 KB
// a staged population (load_raw is a global-only read: not for the ring)
__device__ __forceinline__ float ring_load(const float *row, int x) { return row[x]; }
__device__ __forceinline__ float ring_load(const __half *row, int x) { return __half2float(row[x]); }
// one row (x = 0 .. nx-1) of link i at (y, z) of realization r into dst
__device__ __forceinline__ void tma_row(void *dst, const CUtensorMap *map, int y, int z, int i, int r, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(y), "r"(z), "r"(i), "r"(r), "r"(smem_addr(bar))
        : "memory");
}

template <int PREC, int MODE>
__global__ void __launch_bounds__(TMA_THREADS) k_stream_collide_tma(const Sim S, const __grid_constant__ CUtensorMap tmA,
                                                                     const void *__restrict__ Av, void *__restrict__ Bv,
                                                                     const int groups) {
    using T = typename PopT<PREC>::T;
    constexpr int STAGES = TmaStages<PREC>::n;
    extern __shared__ __align__(128) unsigned char tsm[];
    __shared__ uint64_t bars[STAGES];
    __shared__ int s_abort;
    const int nx = S.nx, ny = S.ny, nz = S.nz;
    const int rows = TMA_THREADS / nx;  // rows per group
    const uint32_t row_bytes = (uint32_t)nx * sizeof(T);
    // a tensor copy lands on a 128-byte boundary: each staged row takes a
    // multiple of 128 bytes, and the ring starts on the first such boundary
    // of the dynamic shared memory (the launch adds 128 bytes for that)
    const uint32_t row_elems = ((row_bytes + 127u) & ~127u) / (uint32_t)sizeof(T);
    const uint32_t stage_elems = (uint32_t)Q * rows * row_elems;
    const int r = blockIdx.y;  // the realization: a CTA's rows are all of one
    const long long total_rows = (long long)nz * ny;
    const long long n_groups = (total_rows + rows - 1) / rows;
    const long long g0 = (long long)blockIdx.x * groups;
    const int ng = (int)max(0ll, min((long long)groups, n_groups - g0));
    const uint32_t ns = (uint32_t)S.ps;
    T *const ring = reinterpret_cast<T *>(tsm + ((128u - (smem_addr(tsm) & 127u)) & 127u));
    const int tid = threadIdx.x;
    const int j = tid / nx, x = tid - j * nx;  // this thread's row in a group and its x
    const bool lane_ok = j < rows;
    float am = 0.f, ax = 0.f, ay = 0.f, az = 0.f;
    const float om = S.omega;
    const float g0f = S.g[0], g1f = S.g[1], g2f = S.g[2];
    const bool has_g = (g0f != 0.f) || (g1f != 0.f) || (g2f != 0.f);
    constexpr float up = PopScale<PREC>::up, down = PopScale<PREC>::down;
    const int xv0 = (x == 0 ? nx - 1 : x - 1), xv2 = (x == nx - 1 ? 0 : x + 1);

    // issue the copies of group k (of this CTA) into its stage
    auto issue = [&](int k) {
        const int st = k % STAGES;
        const long long R0 = (g0 + k) * rows;
        const int nrow = (int)min((long long)rows, total_rows - R0);
        mbar_expect_tx(&bars[st], (uint32_t)nrow * Q * row_bytes);
        for (int jj = 0; jj < nrow; ++jj) {
            const long long R = R0 + jj;
            const int y = (int)(R % ny), z = (int)(R / ny);
            const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
            const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int sy = cy(i) == 1 ? ym : (cy(i) == -1 ? yp : y);
                const int sz = cz(i) == 1 ? zm : (cz(i) == -1 ? zp : z);
                tma_row(ring + (size_t)st * stage_elems + ((size_t)i * rows + jj) * row_elems, &tmA, sy, sz, i, r,
                        &bars[st]);
            }
        }
    };

    if (tid == 0) {
        for (int st = 0; st < STAGES; ++st) mbar_init(&bars[st], 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (S.wait_probe) {
        // test of the bounded wait: stage 0's first phase, which nothing
        // completes (no copy has been issued), runs out after 1 ms
        if (tid == 0 && !mbar_wait(&bars[0], 0u, 1000000ull)) atomicOr(&S.ctrl->status, ST_TIMEOUT);
        return;
    }
    if (tid == 0)
        for (int k = 0; k < min(STAGES, ng); ++k) issue(k);
    int k = 0;
    for (; k < ng; ++k) {
        const int st = k % STAGES;
        const uint32_t par = (uint32_t)((k / STAGES) & 1);
        const bool ready = mbar_wait(&bars[st], par);
        if (!ready) {
            atomicOr(&S.ctrl->status, ST_TIMEOUT);
            s_abort = 1;
        }
        const long long R = (g0 + k) * rows + j;
        if (ready && lane_ok && R < total_rows) {
            const int y = (int)(R % ny), z = (int)(R / ny);
            const int s = x + nx * (y + ny * z);
            const T *A = reinterpret_cast<const T *>(Av) + (size_t)r * Q * ns;
            T *B = reinterpret_cast<T *>(Bv) + (size_t)r * Q * ns;
            const T *row = ring + (size_t)st * stage_elems + (size_t)j * row_elems;  // link i: + i * rows * row_elems
            uint32_t lm = 0u;
            if (S.tileflag[(x >> 5) + S.nxt * (y + ny * z)]) lm = __ldg(S.link + s);
            if (!(lm & SOLID_BIT)) {
                float h[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const int sx = cx(i) == 1 ? xv0 : (cx(i) == -1 ? xv2 : x);
                    h[i] = ((lm >> i) & 1u) ? load_raw(A, (uint32_t)opp(i) * ns + (uint32_t)s)
                                            : ring_load(row + (size_t)i * rows * row_elems, sx);
                }
                float hr[Q], drho_s, jx, jy, jz, rho;
                bgk_relax<PREC>(h, om, hr, drho_s, jx, jy, jz, rho);
                if (MODE != 0 && x >= S.own_lo && x < S.own_hi) {
                    am += drho_s * down; ax += jx * down; ay += jy * down; az += jz * down;
                }
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    float hn = hr[i];
                    if (has_g)
                        hn += up * (3.0f * wq(i) * ((float)cx(i) * g0f + (float)cy(i) * g1f + (float)cz(i) * g2f));
                    store_raw(B, (uint32_t)i * ns + (uint32_t)s, hn);
                }
            }
        }
        __syncthreads();  // every thread is done with stage st (and s_abort is seen by all)
        if (s_abort) break;
        if (tid == 0 && k + STAGES < ng) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(k + STAGES);
        }
    }
    if (s_abort) {
        // copies still in flight land before the CTA's shared memory is released
        if (tid == 0)
            for (int kk = k; kk < min(ng, k + STAGES); ++kk)
                mbar_wait(&bars[kk % STAGES], (uint32_t)((kk / STAGES) & 1));
        return;
    }
    if (MODE != 0) block_partial4(am, ax, ay, az, S.fsum + 4 * (size_t)r, &S.ctrl->status);
}

static size_t tma_smem(const Sim &S) {
    const int esz = S.precision == LBMD_FP16DEV ? 2 : 4;
    const int stages = S.precision == LBMD_FP16DEV ? TmaStages<1>::n : TmaStages<0>::n;
    const size_t row = ((size_t)S.nx * esz + 127) & ~(size_t)127;  // 128-byte rows
    return (size_t)stages * Q * (TMA_THREADS / S.nx) * row + 128;   // + the alignment of the ring
}

// rows of at most 256 sites and a multiple of 16 bytes, a ring within the
// 227 KB a CTA may hold, no thermal noise (the noise needs each site's counter)
bool tma_lattice_ok(const Sim &S) {
    const int esz = S.precision == LBMD_FP16DEV ? 2 : 4;
    return !S.fluct && S.nx >= 1 && S.nx <= TMA_THREADS && (S.nx * esz) % 16 == 0 && tma_smem(S) <= 227u * 1024u;
}

// grant the kernel its shared memory once (not inside a stream capture)
cudaError_t prepare_stream_collide_tma(const Sim &S) {
    const int smem = (int)tma_smem(S);
    cudaError_t e = cudaSuccess;
    if (S.precision == LBMD_FP16DEV) {
        e = cudaFuncSetAttribute(k_stream_collide_tma<1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_stream_collide_tma<1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    } else {
        e = cudaFuncSetAttribute(k_stream_collide_tma<0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_stream_collide_tma<0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    }
    return e;
}

cudaError_t launch_stream_collide_tma(const Sim &S, const CUtensorMap &tmA, const void *A, void *B, int groups,
                                      bool diag, cudaStream_t st) {
    if (!tma_lattice_ok(S) || groups < 1) return cudaErrorInvalidValue;
    const long long total_rows = (long long)S.nz * S.ny;  // per realization
    const int rows = TMA_THREADS / S.nx;
    const long long n_groups = (total_rows + rows - 1) / rows;
    const dim3 grid((unsigned)((n_groups + groups - 1) / groups), S.n_real);
    const size_t smem = tma_smem(S);
#define TMA_LAUNCH(P, M) k_stream_collide_tma<P, M><<<grid, TMA_THREADS, smem, st>>>(S, tmA, A, B, groups)
    if (S.precision == LBMD_FP16DEV) {
        if (diag) TMA_LAUNCH(1, 1); else TMA_LAUNCH(1, 0);
    } else {
        if (diag) TMA_LAUNCH(0, 1); else TMA_LAUNCH(0, 0);
    }
#undef TMA_LAUNCH
    return cudaGetLastError();
}

static dim3 sc_grid(const Sim &S, int by, int zc, int *nzb) {
    *nzb = (S.nz + zc - 1) / zc;
    return dim3((S.nx + 31) / 32, (S.ny + by - 1) / by, (*nzb) * S.n_real);
}

int sc_blocks(const Sim &S, int by, int zc) {
    int nzb;
    dim3 g = sc_grid(S, by, zc, &nzb);
    return (int)(g.x * g.y * g.z);
}

cudaError_t launch_stream_collide(const Sim &S, const void *A, void *B, int by, int zc, bool diag,
                                  cudaStream_t st) {
    int nzb;
    dim3 grid = sc_grid(S, by, zc, &nzb);
    dim3 block(32, by);
    // One site per thread and z-iteration: walking two z sites at a time
    // doubled the loads in flight but needed ~128 registers and lost at
    // every tile shape on GB300.
#define SC_LAUNCH(P, M, F) k_stream_collide<P, M, 1, F><<<grid, block, 0, st>>>(S, A, B, zc, nzb)
    const bool fl = S.fluct != 0;
    if (S.precision == LBMD_FP16DEV) {
        if (diag) { if (fl) SC_LAUNCH(1, 1, true); else SC_LAUNCH(1, 1, false); }
        else { if (fl) SC_LAUNCH(1, 0, true); else SC_LAUNCH(1, 0, false); }
    } else {
        if (diag) { if (fl) SC_LAUNCH(0, 1, true); else SC_LAUNCH(0, 1, false); }
        else { if (fl) SC_LAUNCH(0, 0, true); else SC_LAUNCH(0, 0, false); }
    }
#undef SC_LAUNCH
    return cudaGetLastError();
}

cudaError_t launch_fluid_observables(const Sim &S, const void *A, cudaStream_t st) {
    int nzb;
    const int by = 8, zc = 4;
    dim3 grid = sc_grid(S, by, zc, &nzb);
    dim3 block(32, by);
    if (S.precision == LBMD_FP16DEV) k_stream_collide<1, 2, 2, false><<<grid, block, 0, st>>>(S, A, nullptr, zc, nzb);
    else k_stream_collide<0, 2, 2, false><<<grid, block, 0, st>>>(S, A, nullptr, zc, nzb);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Source pass (Sec. II, Eq. 9 with beta = 3): at every lattice site a bead
// touched this step, f*_i += 3 w_i G.c_i with G the momentum the beads handed
// to the fluid there; G is then cleared.  Sites are found through the list of
// (bead, corner) pairs; the first pair to stamp a site with this step's tag
// applies its source.  Thread r also completes realization r's diagnostics
// row with the fluid sums of the step's lattice pass.  The last block to
// finish advances the step counter.
// ---------------------------------------------------------------------------
template <int PREC>
__global__ void __launch_bounds__(256) k_source(const Sim S, void *__restrict__ Bv) {
    using T = typename PopT<PREC>::T;
    const long long step = S.ctrl->step;
    const int tag = (int)(step & 0x3fffffffll) + 1;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < 8 * S.total_beads) {
        const int gnode = S.pair_node[k];
        if (gnode >= 0) {
            const int r = gnode / S.ns;
            const int s = gnode - r * S.ns;
            const size_t ns = (size_t)S.ns;
            unsigned long long *Gr = S.G + (size_t)r * 3 * ns + s;
            T *B = reinterpret_cast<T *>(Bv) + (size_t)r * Q * S.ps;
            // G and the 19 populations are loaded before the stamp decides
            // whether this pair applies the source, so that all of them and
            // the exchange travel together; a pair that loses the stamp
            // drops what it loaded
            const long long g0 = (long long)__ldcg(Gr), g1 = (long long)__ldcg(Gr + ns), g2 = (long long)__ldcg(Gr + 2 * ns);
            float h[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) h[i] = load_dev_cg(B, (uint32_t)i * (uint32_t)S.ps + (uint32_t)s);
            if (atomicExch(S.stamp + gnode, tag) != tag) {
                const float G0 = (float)g0 * FIX_INV_SCALE_F;
                const float G1 = (float)g1 * FIX_INV_SCALE_F;
                const float G2 = (float)g2 * FIX_INV_SCALE_F;
                Gr[0] = 0ull; Gr[ns] = 0ull; Gr[2 * ns] = 0ull;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const float src = 3.0f * wq(i) * ((float)cx(i) * G0 + (float)cy(i) * G1 + (float)cz(i) * G2);
                    store_dev(B, (uint32_t)i * (uint32_t)S.ps + (uint32_t)s, h[i] + src);
                }
            }
        }
    }
    // the lattice pass of this step has finished: thread r writes the fluid
    // part of realization r's diagnostics row and clears its accumulator
    if (k < S.n_real) {
        long long *acc = S.fsum + 4 * (size_t)k;
        const double unit = fix_unit(FIXD_FLUID);
        lbmd_diag *row = S.ring + (size_t)k * LBMD_DIAG_RING + (step % LBMD_DIAG_RING);
        row->step = step;
        row->mass = S.n_fluid + (double)acc[0] * unit;
        row->p_fluid[0] = (double)acc[1] * unit;
        row->p_fluid[1] = (double)acc[2] * unit;
        row->p_fluid[2] = (double)acc[3] * unit;
        acc[0] = 0; acc[1] = 0; acc[2] = 0; acc[3] = 0;
    }
    // Every thread has used the step it read before this barrier, so the
    // last block's update cannot reach an earlier read; the stores above are
    // for later kernels, which the kernel boundary orders.  No fence.
    __shared__ int am_last;
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(&S.ctrl->src_done, 1u) == gridDim.x - 1u);
    __syncthreads();
    if (am_last && threadIdx.x == 0) {
        S.ctrl->src_done = 0u;
        S.ctrl->step = step + 1;
    }
}

cudaError_t launch_source(const Sim &S, void *B, cudaStream_t st) {
    const int threads = 256;
    const int blocks = max(1, (max(8 * S.total_beads, S.n_real) + threads - 1) / threads);
    if (S.precision == LBMD_FP16DEV) k_source<1><<<blocks, threads, 0, st>>>(S, B);
    else k_source<0><<<blocks, threads, 0, st>>>(S, B);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// state transfer.  The fp32 staging area holds either full populations f
// (host-visible format) or deviations h = f - w (DEV); conversions between the
// two use the exact weights in double precision.
// ---------------------------------------------------------------------------
template <int PREC>
__global__ void k_init_rest(const Sim S, void *Av) {
    using T = typename PopT<PREC>::T;
    const size_t ns = (size_t)S.ns;
    const size_t total = ns * S.n_real;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const size_t r = t / ns, s = t - r * ns;
        T *A = reinterpret_cast<T *>(Av) + r * Q * (size_t)S.ps;
#pragma unroll
        for (int i = 0; i < Q; ++i) store_dev(A, (uint32_t)(i * (size_t)S.ps + s), 0.0f);
    }
}

cudaError_t launch_init_rest(const Sim &S, void *A, cudaStream_t st) {
    if (S.precision == LBMD_FP16DEV) k_init_rest<1><<<4 * 152, 256, 0, st>>>(S, A);
    else k_init_rest<0><<<4 * 152, 256, 0, st>>>(S, A);
    return cudaGetLastError();
}

// rho, ux, uy, uz in staging rows 15..18 -> deviations of f_eq(rho, u) (Eq. 5)
// in rows 0..18
__global__ void k_feq_to_staging(const Sim S, float *stg) {
    const size_t ns = (size_t)S.ns;
    const size_t total = ns * S.n_real;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const size_t r = t / ns, s = t - r * ns;
        float *f = stg + r * Q * ns + s;
        const double rho = f[15 * ns], ux = f[16 * ns], uy = f[17 * ns], uz = f[18 * ns];
        const bool sol = S.solid[s] != 0;
        const double usq = 1.5 * (ux * ux + uy * uy + uz * uz);
        float out[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double cu = 3.0 * (cx(i) * ux + cy(i) * uy + cz(i) * uz);
            out[i] = sol ? 0.0f : (float)(wq_exact(i) * ((rho - 1.0) + rho * (cu + 0.5 * cu * cu - usq)));
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i * ns] = out[i];
    }
}

cudaError_t launch_feq_to_staging(const Sim &S, float *staging, cudaStream_t st) {
    k_feq_to_staging<<<4 * 152, 256, 0, st>>>(S, staging);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// State transfer between the populations and the fp32 staging area
// [realization][19][site], with f = w_i + h at the host.  The conversions
// round as the FP64 expressions float(double(h) + w_i) and
// float(double(f) - w_i) do (w_i the double nearest the weight), without FP64
// arithmetic in all but rare cases: FP64 runs at a small fraction of the FP32
// rate on this GPU, and with 19 conversions per site in FP64 a transfer of the
// 4.19M-site lattice took 444 us (1.4 TB/s); in FP32 it takes 179-197 us.
//
// The double constant cd is the exact sum of three floats c0 + c1 + c2.  Two
// error-free sums (TwoSum, Knuth) give r = RN32(v + c0 + c1) and the exact
// remainder, so v + cd = r + rho exactly, rho = d + et + c2 (computed in FP32,
// within `bound`).  RN64 moves v + cd by at most 2^-53 |v + cd|.  When
// |rho| stays below half an ulp of r by more than both, RN32(RN64(v + cd)) = r;
// when r is zero, tiny, a power of two (unequal gaps), not finite, or rho is
// near the midpoint, the FP64 expression is evaluated instead.
// ---------------------------------------------------------------------------
struct WSplit { float c0, c1, c2; };
__host__ __device__ constexpr WSplit wsplit(double cd) {
    return {(float)cd, (float)(cd - (double)(float)cd),
            (float)(cd - (double)(float)cd - (double)(float)(cd - (double)(float)cd))};
}

// the FP64 expression itself, out of line: evaluated only where the fast
// path cannot decide (inline, the compiler may evaluate it for every element
// and select, which costs the FP64 rate the fast path avoids)
__device__ __noinline__ float add_double_rn_fp64(float v, double cd) { return (float)((double)v + cd); }

// float(double(v) + cd) for cd = W.c0 + W.c1 + W.c2
__device__ __forceinline__ float add_double_rn(float v, WSplit W, double cd) {
    float s, e, t, et, r, d;
    two_sum(v, W.c0, s, e);
    two_sum(e, W.c1, t, et);
    two_sum(s, t, r, d);
    const float rho = (d + et) + W.c2;
    const float bound = fmaf(fabsf(d) + fabsf(et) + fabsf(W.c2), 0x1p-22f, fabsf(r) * 0x1p-50f);
    const uint32_t rb = __float_as_uint(r), eb = rb & 0x7f800000u;
    const bool fast = eb >= (25u << 23) && eb != 0x7f800000u && (rb & 0x007fffffu) != 0u &&
                      fmaf(__uint_as_float(eb), 0x1p-24f, -fabsf(rho)) > bound;
    if (!fast) r = add_double_rn_fp64(v, cd);
    return r;
}

template <int I>
__device__ __forceinline__ float plus_weight(float h) {  // float(double(h) + w_I)
    constexpr double cd = wq_exact(I);
    constexpr WSplit W = wsplit(cd);
    return add_double_rn(h, W, cd);
}
template <int I>
__device__ __forceinline__ float minus_weight(float f) {  // float(double(f) - w_I)
    constexpr double cd = -wq_exact(I);
    constexpr WSplit W = wsplit(cd);
    return add_double_rn(f, W, cd);
}

// The 19 loads of a site are issued before any of its stores, so that they
// are in flight together (the compiler may not move a load above a store to
// a buffer it cannot tell apart).
template <int I, int PREC>
__device__ __forceinline__ float pull_load(const typename PopT<PREC>::T *A, uint32_t lm, int x, int y, int z, uint32_t s,
                                           const Sim &S) {
    if (lm & SOLID_BIT) return 0.0f;
    const uint32_t ps = (uint32_t)S.ps;
    const uint32_t idx = ((lm >> I) & 1u) ? (uint32_t)opp(I) * ps + s
                                           : (uint32_t)I * ps + (uint32_t)(wrapi(x - cx(I), S.nx) +
                                                                          S.nx * (wrapi(y - cy(I), S.ny) + S.ny * wrapi(z - cz(I), S.nz)));
    return load_dev(A, idx);
}

template <int I>
__device__ __forceinline__ float push_load(const float *f, uint32_t lm, int x, int y, int z, uint32_t s, const Sim &S) {
    if (lm & SOLID_BIT) return 0.0f;
    const bool bb = (lm >> opp(I)) & 1u;  // y + c_I is solid: the link comes back as opp(I)
    const uint32_t src = bb ? s : (uint32_t)(wrapi(x + cx(I), S.nx) + S.nx * (wrapi(y + cy(I), S.ny) + S.ny * wrapi(z + cz(I), S.nz)));
    return __ldg(f + (size_t)(bb ? opp(I) : I) * S.ns + src);
}

template <int PREC, bool DEV, int... I>
__device__ __forceinline__ void pull_site(const typename PopT<PREC>::T *A, float *f, uint32_t lm, int x, int y, int z,
                                          uint32_t s, const Sim &S, std::integer_sequence<int, I...>) {
    float h[Q];
    ((h[I] = pull_load<I, PREC>(A, lm, x, y, z, s, S)), ...);
    const bool solid = lm & SOLID_BIT;
    ((f[(size_t)I * S.ns + s] = solid ? 0.0f : (DEV ? h[I] : plus_weight<I>(h[I]))), ...);
}
template <int PREC, bool DEV, int... I>
__device__ __forceinline__ void push_site(const float *f, typename PopT<PREC>::T *A, uint32_t lm, int x, int y, int z,
                                          uint32_t s, const Sim &S, std::integer_sequence<int, I...>) {
    float v[Q];
    ((v[I] = push_load<I>(f, lm, x, y, z, s, S)), ...);
    const bool solid = lm & SOLID_BIT;
    (store_dev(A, (uint32_t)I * (uint32_t)S.ps + s, solid ? 0.0f : (DEV ? v[I] : minus_weight<I>(v[I]))), ...);
}

// pulled populations f^n (what the next step starts from) -> staging; one
// thread per site, realization blockIdx.y
template <int PREC, bool DEV>
__global__ void __launch_bounds__(256) k_pull_to_staging(const Sim S, const void *Av, float *stg) {
    using T = typename PopT<PREC>::T;
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= (uint32_t)S.ns) return;
    const int r = blockIdx.y;
    const uint32_t nxy = (uint32_t)S.nx * (uint32_t)S.ny;
    const int z = (int)(s / nxy), rem = (int)(s - (uint32_t)z * nxy), y = rem / S.nx, x = rem - y * S.nx;
    pull_site<PREC, DEV>(reinterpret_cast<const T *>(Av) + (size_t)r * Q * S.ps, stg + (size_t)r * Q * S.ns, S.link[s],
                         x, y, z, s, S, std::make_integer_sequence<int, Q>{});
}

cudaError_t launch_pull_to_staging(const Sim &S, const void *A, float *staging, bool dev, cudaStream_t st) {
    const dim3 grid((unsigned)((S.ns + 255) / 256), (unsigned)S.n_real);
    if (S.precision == LBMD_FP16DEV) {
        if (dev) k_pull_to_staging<1, true><<<grid, 256, 0, st>>>(S, A, staging);
        else k_pull_to_staging<1, false><<<grid, 256, 0, st>>>(S, A, staging);
    } else {
        if (dev) k_pull_to_staging<0, true><<<grid, 256, 0, st>>>(S, A, staging);
        else k_pull_to_staging<0, false><<<grid, 256, 0, st>>>(S, A, staging);
    }
    return cudaGetLastError();
}

// inverse of the pull: A_i(y) = f_i(y + c_i), or f_opp(i)(y) when y + c_i is solid
template <int PREC, bool DEV>
__global__ void __launch_bounds__(256) k_push_from_staging(const Sim S, const float *stg, void *Av) {
    using T = typename PopT<PREC>::T;
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= (uint32_t)S.ns) return;
    const int r = blockIdx.y;
    const uint32_t nxy = (uint32_t)S.nx * (uint32_t)S.ny;
    const int z = (int)(s / nxy), rem = (int)(s - (uint32_t)z * nxy), y = rem / S.nx, x = rem - y * S.nx;
    push_site<PREC, DEV>(stg + (size_t)r * Q * S.ns, reinterpret_cast<T *>(Av) + (size_t)r * Q * S.ps, S.link[s],
                         x, y, z, s, S, std::make_integer_sequence<int, Q>{});
}

cudaError_t launch_push_from_staging(const Sim &S, const float *staging, void *A, bool dev, cudaStream_t st) {
    const dim3 grid((unsigned)((S.ns + 255) / 256), (unsigned)S.n_real);
    if (S.precision == LBMD_FP16DEV) {
        if (dev) k_push_from_staging<1, true><<<grid, 256, 0, st>>>(S, staging, A);
        else k_push_from_staging<1, false><<<grid, 256, 0, st>>>(S, staging, A);
    } else {
        if (dev) k_push_from_staging<0, true><<<grid, 256, 0, st>>>(S, staging, A);
        else k_push_from_staging<0, false><<<grid, 256, 0, st>>>(S, staging, A);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Slab mode: copy `planes` consecutive local x planes from x_first on between
// the populations and a plane buffer [19][planes][nz][ny] (raw storage
// values), into the buffer (to_buf) or out of it.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_slab_planes(const Sim S, T *pop, T *buf, int x_first, int planes, bool to_buf) {
    const size_t nyz = (size_t)S.ny * S.nz;
    const size_t total = (size_t)Q * planes * nyz;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const size_t i = t / (planes * nyz), rem = t - i * planes * nyz;
        const size_t p = rem / nyz, zy = rem - p * nyz;
        const size_t z = zy / S.ny, y = zy - z * S.ny;
        T *site = pop + i * (size_t)S.ps + (size_t)(x_first + (int)p) + (size_t)S.nx * (y + (size_t)S.ny * z);
        if (to_buf) buf[t] = *site;
        else *site = buf[t];
    }
}

cudaError_t launch_slab_planes(const Sim &S, void *pop, void *buf, int x_first, int planes, bool to_buf,
                               cudaStream_t st) {
    const size_t total = (size_t)Q * planes * S.ny * S.nz;
    const int blocks = (int)min((total + 255) / 256, (size_t)4 * 152);
    if (S.precision == LBMD_FP16DEV)
        k_slab_planes<__half><<<blocks, 256, 0, st>>>(S, (__half *)pop, (__half *)buf, x_first, planes, to_buf);
    else
        k_slab_planes<float><<<blocks, 256, 0, st>>>(S, (float *)pop, (float *)buf, x_first, planes, to_buf);
    return cudaGetLastError();
}

}  // namespace lbmd
