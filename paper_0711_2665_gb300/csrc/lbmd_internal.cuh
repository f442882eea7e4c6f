// lbmd_internal.cuh -- device-side definitions shared by the kernels of the
// coupled LB-MD library (not part of the public ABI).
//
// Data layout in HBM (one device buffer owned by the caller):
//   populations  A, B      [n_real][19][ps]  fp32, or fp16 deviations (f - w) * 2^12
//                          A holds the post-collision populations f* of the last
//                          step; the next step pulls from A and writes B.
//   staging                [n_real][19][ns]  fp32 host-transfer area
//   link                   [ns] u32: bit i set = the pull of link i bounces back
//                          (its source x - c_i is solid); bit 31 = site solid
//   tileflag               [nxt][ny][nz] u8: 1 if any of the 32 sites of the x-tile
//                          has a bounce-back link or is solid (warp-uniform fast path)
//   solid                  [ns] u8
//   G                      [n_real][3][ns] i64 fixed point (2^40): momentum handed
//                          to the fluid by the beads this step
//   stamp                  [n_real][ns] i32: last step a source was applied at a site
//   beads                  float4 r_hi, r_lo (unwrapped position as a float-float
//                          pair), v, up, J  [total_beads]
//   pair_node              [total_beads][8] i32: global site of each fluid corner
//   partial / ring / ctrl  reduction scratch, per-step diagnostics, counters
#pragma once

#include <cuda.h>  // CUtensorMap and its enums (no driver library is linked)
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/lbmd.h"

namespace lbmd {

// ---------------------------------------------------------------------------
// D3Q19 (Sec. II).  Order: rest, +x,-x,+y,-y,+z,-z, then the 12 face diagonals
// in opposite pairs.  Compile-time tables so that unrolled loops fold them.
// ---------------------------------------------------------------------------
constexpr int Q = 19;
__host__ __device__ constexpr int cx(int i) {
    return i == 1 || i == 7 || i == 9 || i == 11 || i == 13 ? 1
         : i == 2 || i == 8 || i == 10 || i == 12 || i == 14 ? -1 : 0;
}
__host__ __device__ constexpr int cy(int i) {
    return i == 3 || i == 7 || i == 10 || i == 15 || i == 17 ? 1
         : i == 4 || i == 8 || i == 9 || i == 16 || i == 18 ? -1 : 0;
}
__host__ __device__ constexpr int cz(int i) {
    return i == 5 || i == 11 || i == 14 || i == 15 || i == 18 ? 1
         : i == 6 || i == 12 || i == 13 || i == 16 || i == 17 ? -1 : 0;
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr float wq(int i) {
    return i == 0 ? (1.0f / 3.0f) : (i <= 6 ? (1.0f / 18.0f) : (1.0f / 36.0f));
}

// Mode k of the D3Q19 moment basis on velocity c_i (orthogonal under the
// weights): 0 density, 1-3 momentum, 4-9 stress (bulk, two normal-stress
// differences, three shear), 10-18 ghost modes.  Used by the fluctuating LB.
__host__ __device__ constexpr float mode_e(int k, int i) {
    return k == 0 ? 1.0f
         : k == 1 ? (float)cx(i)
         : k == 2 ? (float)cy(i)
         : k == 3 ? (float)cz(i)
         : k == 4 ? (float)(cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i) - 1)
         : k == 5 ? (float)(3 * cx(i) * cx(i) - (cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i)))
         : k == 6 ? (float)(cy(i) * cy(i) - cz(i) * cz(i))
         : k == 7 ? (float)(cx(i) * cy(i))
         : k == 8 ? (float)(cy(i) * cz(i))
         : k == 9 ? (float)(cz(i) * cx(i))
         : k == 10 ? (float)((3 * (cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i)) - 5) * cx(i))
         : k == 11 ? (float)((3 * (cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i)) - 5) * cy(i))
         : k == 12 ? (float)((3 * (cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i)) - 5) * cz(i))
         : k == 13 ? (float)((cy(i) * cy(i) - cz(i) * cz(i)) * cx(i))
         : k == 14 ? (float)((cz(i) * cz(i) - cx(i) * cx(i)) * cy(i))
         : k == 15 ? (float)((cx(i) * cx(i) - cy(i) * cy(i)) * cz(i))
         : k == 16 ? (float)(3 * (cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i)) * (cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i))
                             - 6 * (cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i)) + 1)
         : k == 17 ? (float)((2 * (cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i)) - 3) *
                             (3 * cx(i) * cx(i) - (cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i))))
         : k == 18 ? (float)((2 * (cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i)) - 3) * (cy(i) * cy(i) - cz(i) * cz(i)))
         : 0.0f;
}

constexpr uint32_t SOLID_BIT = 0x80000000u;
// set on a site when a solid site lies within Chebyshev distance
// near_solid_radius (computed on the host from the wall-list radius): a bead
// whose cell corner lacks it has no solid site in its wall-list box
constexpr uint32_t NEAR_SOLID_BIT = 0x40000000u;
constexpr float FP16_SCALE = 4096.0f;          // 2^12
constexpr float FP16_INV_SCALE = 1.0f / 4096.0f;
constexpr double FIX_SCALE = 1099511627776.0;  // 2^40
constexpr float FIX_SCALE_F = 1099511627776.0f;

// Fixed-point scales (powers of two) of the per-step diagnostics sums.  The
// sums are 64-bit integer sums: exact, and the same in any order and for any
// launch shape.  Ranges: |sum of rho - 1| and |sum of rho u| over one
// realization below 2^22; bead |v| below 2^12; unwrapped |x| below 2^15;
// distances from a part's centroid below 2^10.
constexpr int FIXD_FLUID = 40;  // rho - 1 and rho u
constexpr int FIXD_V = 40;      // bead velocities and work rates
constexpr int FIXD_X = 36;      // bead positions
constexpr int FIXD_D2 = 30;     // squared distances from a centroid

// round(x 2^S) as a 64-bit integer, with integer operations only (the
// hardware conversion runs on the slow double-precision path of this GPU).
// Halves round away from zero; zero, subnormal and non-finite x give 0 (the
// callers flag non-finite values themselves).
__device__ __forceinline__ long long fix_of(float x, int S) {
    const unsigned b = __float_as_uint(x);
    const int e = (int)((b >> 23) & 0xffu);
    if (e == 0 || e == 0xff) return 0;
    const long long m = (long long)((b & 0x7fffffu) | 0x800000u);
    const int sh = e - 150 + S;  // x 2^S = m 2^sh
    long long r = 0;
    if (sh >= 0) r = m << min(sh, 39);
    else if (sh > -25) r = (m + (1ll << (-sh - 1))) >> (-sh);
    return (b >> 31) ? -r : r;
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// 2^-S as a double (exact)
__host__ __device__ constexpr double fix_unit(int S) { return S <= 0 ? 1.0 : 0.5 * fix_unit(S - 1); }
constexpr float FIX_INV_SCALE_F = 1.0f / 1099511627776.0f;

constexpr int MAX_CLUSTER = 16;  // blocks per chain (above 8: non-portable cluster size)
constexpr int NBR_CAP = 32;     // bead-bead neighbours per bead
constexpr int WALL_CAP = 12;    // solid sites within the wall-list radius per bead
constexpr int HASH_SIZE = 2048; // cell hash slots (>= 2 * max beads per realization)
constexpr int BRUTE_MAX = 512;  // chains up to this length build pair lists without the hash

// status bits latched in Ctrl::status
constexpr int ST_NONFINITE = 1;
constexpr int ST_CAPACITY = 2;
constexpr int ST_TIMEOUT = 4;

struct Ctrl {
    long long step;          // LB step counter = Philox counter
    int status;              // ST_* bits
    unsigned int src_done;   // blocks finished (source kernel; last one advances step)
    int pad[2];
};

// Everything a kernel needs, passed by value.
struct Sim {
    // lattice
    int nx, ny, nz, ns, nxt, n_real;
    int ps;  // stride between population arrays: ns rounded up to 64
    uint32_t real_base;  // global index of realization 0 (noise key)
    int interp;          // 0 trilinear, 1 nearest grid point
    int integrator;      // 0 velocity Verlet (explicit friction), 1 stochastic position Verlet
    float spv_c, spv_g1, spv_sig;  // exp(-gamma h), (1 - c)/gamma, sqrt(kT (1 - c^2)) over a sub-step h
    int fluct;           // fluctuating LB on
    float fl_amp[15];    // sqrt(3 kT_lb (1 - (1 - omega)^2) / b_k), modes k = 4..18 (times sqrt(rho))
    float inx, iny, inz;     // 1/nx, 1/ny, 1/nz
    int precision;
    float omega;
    float g[3];
    double n_fluid;          // fluid sites per realization
    // beads
    int total_beads, max_beads;
    int wall_x, pore_h, pore_ylo, pore_zlo;
    float k_bond, r0, kappa;
    float lj_eps, lj_sig2, lj_rc2;
    float wall_eps, wall_sig2, wall_rc2;
    float E, gamma, kT;
    int M, Mb;
    int md_T, md_C;          // particle-kernel shape override (0 = automatic)
    int md_pull;             // chain exchange between a cluster's blocks: 0 push, 1 pull (halo)
    int md_bw;               // bonded terms: 0 automatic, 1 by every bead's lanes, 2 by a block's last warp
    int md_reserve;          // 1: the particle kernel's blocks claim their SMs' whole shared memory
    int smem_optin;          // the device's opt-in shared memory per block (bytes)
    int wait_probe;          // test of the bounded waits: the tensor-copy lattice pass waits on a barrier
                             // nothing completes (1 ms), before any copy, and latches ST_TIMEOUT
    // The beads' frame.  Bead positions live in the whole lattice (bnx along
    // x); the populations of this handle cover nx planes from global x plane
    // gx0 on.  Without slabs bnx = nx, gx0 = 0 and the handle owns every
    // plane.  In slab mode (one lattice split over handles in x) the handle
    // holds its slab's planes [own_lo, own_hi) plus ghost planes, and blink /
    // bwallmask are the whole lattice's geometry for the bead-wall lists.
    int slab;                // 1: this handle is one x-slab of a larger lattice
    int bnx;                 // x extent of the whole lattice
    float binx;              // 1 / bnx
    int gx0;                 // global x of local plane 0
    int own_lo, own_hi;      // local planes this handle owns (sums, the spread, u_p of beads whose cell starts there)
    const uint32_t *blink;   // link words of the whole lattice (NEAR_SOLID_BIT, SOLID_BIT)
    const unsigned long long *bwallmask;  // solid masks of the whole lattice
    // placement of the chains in the particle kernel's clusters: per block
    // (realization or -1, rank within its chain, the chain's blocks, the
    // chain's first rank in the cluster); md_clusters clusters of the shape's C
    const int4 *md_map;
    int md_clusters;
    float skin_half2;       // (skin/2)^2: displacement that forces a list rebuild
    float rl2, rlw2, rlw;    // bead and wall list radii (squared) and wall radius
    int ncell[3];            // cells per axis for the neighbour hash (>= 3 to use it)
    float cell_per_site[3];  // ncell / n per axis
    unsigned long long seed;
    // buffers
    const uint32_t *link;
    const unsigned long long *wallmask;  // [ns] solid sites of the 4x4x4 box from (x-1, y-1, z-1)
    const uint8_t *tileflag;
    const uint8_t *solid;
    unsigned long long *G;
    int *stamp;
    float4 *r_hi, *r_lo, *v, *up, *J;
    float4 *bsnap;           // [3][total_beads] r_hi, r_lo, v at the start of the step (written by the gather)
    int *pair_node;          // [total_beads][8] global site of each fluid corner, -1 if none
    float *pair_w;           // [total_beads][8] normalised trilinear weight
    const int *bead_real;    // [total_beads] realization of each bead
    const int *bead_off;
    long long *fsum;         // [2][n_real][4] fixed-point fluid sums (per-step, observables); zero between uses
    lbmd_diag *ring;         // [n_real][LBMD_DIAG_RING]
    lbmd_obs *obs;           // [n_real]
    lbmd_transloc *tl;       // [n_real] translocation records
    Ctrl *ctrl;
    unsigned long long *phase;  // [PHASES] SM cycles per particle-kernel phase, or null
    // The step's starting Verlet lists (k_lists), per bead: bead-bead pairs
    // within the list radius in ascending order, and solid sites within the
    // wall-list radius
    uint16_t *nbr_g;         // [total_beads][NBR_CAP]
    uint32_t *wal_g;         // [total_beads][WALL_CAP] packed x | y << 12 | z << 22
    int *nn_g, *nw_g;        // [total_beads] list lengths
    // Trajectory record of the MD cycle for the adjoint, or null:
    // traj[slot * total_beads + bead] with the slots of traj_slot_* below
    float4 *traj;
};

// Slots of the MD trajectory record: positions (hi, lo) at the M*Mb + 1
// sub-step boundaries, the velocity before each of the 2M half kicks (w = 1
// when the bead sat in the pore channel), the frozen fluid velocity u_p and
// the impulse J.
__host__ __device__ inline int traj_npos(int M, int Mb) { return M * Mb + 1; }
__host__ __device__ inline int traj_slot_hi(int M, int Mb, int t) { return t; }
__host__ __device__ inline int traj_slot_lo(int M, int Mb, int t) { return traj_npos(M, Mb) + t; }
__host__ __device__ inline int traj_slot_kick(int M, int Mb, int k) { return 2 * traj_npos(M, Mb) + k; }
__host__ __device__ inline int traj_slot_up(int M, int Mb) { return 2 * traj_npos(M, Mb) + 2 * M; }
__host__ __device__ inline int traj_slot_J(int M, int Mb) { return 2 * traj_npos(M, Mb) + 2 * M + 1; }
__host__ __device__ inline int traj_slots(int M, int Mb) { return 2 * traj_npos(M, Mb) + 2 * M + 2; }

// load, lists, md, spread, rebuild cycles inside md, number of rebuilds
constexpr int PHASES = 6;

// ---------------------------------------------------------------------------
// population storage
// ---------------------------------------------------------------------------
// Both precisions store deviations from the rest state, h = f - w (PREC 0:
// fp32 h; PREC 1: fp16 h * 2^12), so the constant w_i is exact by definition
// and rounding is relative to the (small) deviation, not to w_i.
template <int PREC> struct PopT;
template <> struct PopT<0> { using T = float; };
template <> struct PopT<1> { using T = __half; };

// exact weights for host-visible conversions f <-> h
__host__ __device__ constexpr double wq_exact(int i) {
    return i == 0 ? (1.0 / 3.0) : (i <= 6 ? (1.0 / 18.0) : (1.0 / 36.0));
}

__device__ __forceinline__ float load_dev(const float *base, uint32_t idx) { return __ldg(base + idx); }
__device__ __forceinline__ float load_dev(const __half *base, uint32_t idx) {
    return __half2float(__ldg(base + idx)) * FP16_INV_SCALE;
}
// coherent load for data another kernel of the same step may have written
__device__ __forceinline__ float load_dev_cg(const float *base, uint32_t idx) { return __ldcg(base + idx); }
__device__ __forceinline__ float load_dev_cg(const __half *base, uint32_t idx) {
    return __half2float(__ldcg(base + idx)) * FP16_INV_SCALE;
}
__device__ __forceinline__ void store_dev(float *base, uint32_t idx, float h) { base[idx] = h; }
// stored units: h for FP32, h * 2^12 for FP16 (the lattice kernels compute in
// stored units and scale the moments, so no load or store is multiplied)
template <int PREC> struct PopScale;
template <> struct PopScale<0> { static constexpr float up = 1.0f, down = 1.0f; };
template <> struct PopScale<1> { static constexpr float up = FP16_SCALE, down = FP16_INV_SCALE; };
// global memory only (a read-only cached load)
__device__ __forceinline__ float load_raw(const float *base, uint32_t idx) { return __ldg(base + idx); }
__device__ __forceinline__ float load_raw(const __half *base, uint32_t idx) { return __half2float(__ldg(base + idx)); }
__device__ __forceinline__ void store_raw(float *base, uint32_t idx, float v) { base[idx] = v; }
__device__ __forceinline__ void store_raw(__half *base, uint32_t idx, float v) { base[idx] = __float2half_rn(v); }
__device__ __forceinline__ void store_dev(__half *base, uint32_t idx, float h) {
    base[idx] = __float2half_rn(h * FP16_SCALE);
}

// ---------------------------------------------------------------------------
// mbarriers (sm_90 and later).  Every wait is bounded: at most
// MBAR_WAIT_LIMIT polls or MBAR_WAIT_NS ns, after which the caller latches
// ST_TIMEOUT.  An expected phase takes microseconds.
// ---------------------------------------------------------------------------
constexpr unsigned MBAR_WAIT_LIMIT = 1u << 22;
constexpr unsigned long long MBAR_WAIT_NS = 250000000;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// the phase's one arrival, announcing `bytes` of transfers that complete it
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bounded wait for the phase of parity `parity` to complete (at most
// MBAR_WAIT_LIMIT polls or limit_ns); false: gave up
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          unsigned long long limit_ns = MBAR_WAIT_NS) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned k = 0; k < MBAR_WAIT_LIMIT; ++k) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((k & 63u) == 63u && global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the Gaussian mapping
// used for the bead noise: key = (seed_lo, seed_hi ^ realization), counter =
// (bead, step_lo, substep, step_hi); u = (top 24 bits + 1/2) 2^-24; Box-Muller.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ float3 gauss3(unsigned long long seed, uint32_t realization,
                                         uint32_t bead, long long step, uint32_t substep) {
    const uint2 key = make_uint2((uint32_t)(seed & 0xffffffffull), (uint32_t)(seed >> 32) ^ realization);
    const uint4 ctr = make_uint4(bead, (uint32_t)((unsigned long long)step & 0xffffffffull), substep,
                                 (uint32_t)((unsigned long long)step >> 32));
    const uint4 x = philox4x32_10(ctr, key);
    const float u0 = ((float)(x.x >> 8) + 0.5f) * (1.0f / 16777216.0f);
    const float u1 = ((float)(x.y >> 8) + 0.5f) * (1.0f / 16777216.0f);
    const float u2 = ((float)(x.z >> 8) + 0.5f) * (1.0f / 16777216.0f);
    const float u3 = ((float)(x.w >> 8) + 0.5f) * (1.0f / 16777216.0f);
    const float a = sqrtf(-2.0f * logf(u0));
    const float b = sqrtf(-2.0f * logf(u2));
    float s1, c1, s3, c3;
    sincospif(2.0f * u1, &s1, &c1);
    sincospif(2.0f * u3, &s3, &c3);
    return make_float3(a * c1, a * s1, b * c3);
}

// Sixteen standard normals for the fluctuations of one site and step:
// counters (site, step_lo, 0xF0000000 + j, step_hi), j = 0..3, same key as the
// bead noise; Box-Muller on (u0, u1) and (u2, u3) of each call.
__device__ __forceinline__ void fluid_noise16(unsigned long long seed, uint32_t realization, uint32_t site, long long step,
                                              float (&z)[16]) {
    const uint2 key = make_uint2((uint32_t)(seed & 0xffffffffull), (uint32_t)(seed >> 32) ^ realization);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint4 ctr = make_uint4(site, (uint32_t)((unsigned long long)step & 0xffffffffull), 0xF0000000u + (uint32_t)j,
                                     (uint32_t)((unsigned long long)step >> 32));
        const uint4 x = philox4x32_10(ctr, key);
        const float u0 = ((float)(x.x >> 8) + 0.5f) * (1.0f / 16777216.0f);
        const float u1 = ((float)(x.y >> 8) + 0.5f) * (1.0f / 16777216.0f);
        const float u2 = ((float)(x.z >> 8) + 0.5f) * (1.0f / 16777216.0f);
        const float u3 = ((float)(x.w >> 8) + 0.5f) * (1.0f / 16777216.0f);
        const float a = sqrtf(-2.0f * logf(u0)), b = sqrtf(-2.0f * logf(u2));
        float s1, c1, s3, c3;
        sincospif(2.0f * u1, &s1, &c1);
        sincospif(2.0f * u3, &s3, &c3);
        z[4 * j + 0] = a * c1;
        z[4 * j + 1] = a * s1;
        z[4 * j + 2] = b * c3;
        z[4 * j + 3] = b * s3;
    }
}

// ---------------------------------------------------------------------------
// float-float positions: unwrapped coordinate = hi + lo, |lo| <= ulp(hi)/2
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// hi + lo += d: the rounding error of hi + d is carried in lo (renormalised by
// ff_norm once per LB step, so lo stays far below ulp(hi) * steps)
__device__ __forceinline__ void ff_add(float &hi, float &lo, float d) {
    float s, e;
    two_sum(hi, d, s, e);
    hi = s;
    lo += e;
}
__device__ __forceinline__ void ff_norm(float &hi, float &lo) {
    float s, e;
    two_sum(hi, lo, s, e);
    hi = s;
    lo = e;
}
// minimum-image difference of two float-float coordinates on an axis of length
// n (inv = 1/n; a rounding of d * inv can only matter at separations of n/2,
// far beyond every cut-off)
__device__ __forceinline__ float ff_diff(float ahi, float alo, float bhi, float blo, float n, float inv) {
    float d = (ahi - bhi) + (alo - blo);
    return d - n * rintf(d * inv);
}
// wrapped coordinate in [0, n)
__device__ __forceinline__ float ff_wrap(float hi, float lo, float n, float inv) {
    float x = hi - n * floorf(hi * inv);
    if (x < 0.0f) x += n;
    if (x >= n) x -= n;
    x += lo;
    if (x < 0.0f) x += n;
    if (x >= n) x -= n;
    // non-finite or runaway coordinates must never become out-of-range lattice
    // indices: they are pinned to 0 (the step's non-finite check reports them)
    if (!(x >= 0.0f && x < n)) x = 0.0f;
    return x;
}

// atan2(y, x) for y >= 0, branch-free: reduce to t = min/max in [0, 1], then
// atan(t) = t P(t^2) with P the degree-8 fit of atan(t)/t made by
// csrc/fit_atan.py (relative error < 1.1e-7 in fp32), then reflect.
__device__ __forceinline__ float atan_pos(float y, float x) {
    const float ax = fabsf(x);
    const float mx = fmaxf(y, ax), mn = fminf(y, ax);
    const float t = mx > 0.0f ? __fdividef(mn, mx) : 0.0f;
    const float s = t * t;
    float p = 2.903541317e-03f;
    p = fmaf(p, s, -1.628293283e-02f);
    p = fmaf(p, s, 4.303918779e-02f);
    p = fmaf(p, s, -7.533655316e-02f);
    p = fmaf(p, s, 1.065466478e-01f);
    p = fmaf(p, s, -1.420712918e-01f);
    p = fmaf(p, s, 1.999305338e-01f);
    p = fmaf(p, s, -3.333309293e-01f);
    p = fmaf(p, s, 1.0f);
    float a = t * p;
    a = y > ax ? 1.5707963268f - a : a;
    return x < 0.0f ? 3.1415926536f - a : a;
}

// wrap an index that is at most one period outside [0, n)
__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }
// wrap any index into [0, n)
__device__ __forceinline__ int wrap_any(int i, int n) { const int m = i % n; return m < 0 ? m + n : m; }

// Field channel of Sec. IV: |x - wall_x| <= 3/2 (minimum image) and y, z inside the
// pore cross-section padded by half a site.
__device__ __forceinline__ bool in_channel(const Sim &S, float xw, float yw, float zw) {
    if (S.wall_x < 0) return false;
    float dx = xw - (float)S.wall_x;
    dx -= (float)S.bnx * rintf(dx * S.binx);
    if (fabsf(dx) > 1.5f) return false;
    if (yw < (float)S.pore_ylo - 0.5f || yw > (float)(S.pore_ylo + S.pore_h) - 0.5f) return false;
    if (zw < (float)S.pore_zlo - 0.5f || zw > (float)(S.pore_zlo + S.pore_h) - 0.5f) return false;
    return true;
}

// ---------------------------------------------------------------------------
// host-side launchers (defined in the kernel translation units)
// ---------------------------------------------------------------------------
int sc_blocks(const Sim &S, int by, int zc);
cudaError_t launch_stream_collide(const Sim &S, const void *A, void *B, int by, int zc,
                                  bool diag, cudaStream_t st);
// the lattice pass fed by tensor copies (no fluctuations, nx <= 256, rows of
// a multiple of 16 bytes): tmA describes buffer A as a 5-D tensor
// (x, y, z, link, realization) with one-row boxes; groups: row groups per CTA
bool tma_lattice_ok(const Sim &S);
bool x2_lattice_ok(const Sim &S);
cudaError_t launch_stream_collide_x2(const Sim &S, const void *A, void *B, int by, int zc, bool diag,
                                     cudaStream_t st);
cudaError_t prepare_stream_collide_tma(const Sim &S);
cudaError_t launch_stream_collide_tma(const Sim &S, const CUtensorMap &tmA, const void *A, void *B, int groups,
                                      bool diag, cudaStream_t st);
cudaError_t launch_fluid_observables(const Sim &S, const void *A, cudaStream_t st);
cudaError_t launch_source(const Sim &S, void *B, cudaStream_t st);
cudaError_t launch_init_rest(const Sim &S, void *A, cudaStream_t st);
cudaError_t launch_feq_to_staging(const Sim &S, float *staging, cudaStream_t st);
cudaError_t launch_pull_to_staging(const Sim &S, const void *A, float *staging, bool dev, cudaStream_t st);
cudaError_t launch_push_from_staging(const Sim &S, const float *staging, void *A, bool dev, cudaStream_t st);
cudaError_t launch_slab_planes(const Sim &S, void *pop, void *buf, int x_first, int planes, bool to_buf,
                               cudaStream_t st);
// launch shape of the particle kernel: T threads per bead, clusters of C
// blocks per realization, Nc beads per block
struct MdShape {
    int T, C, Nc, threads;
    bool bw;  // bonded terms by a block's last warp
    size_t smem;         // shared memory the kernel uses
    size_t launch_smem;  // shared memory a block is launched with (smem, or the opt-in maximum when reserving,
                         // less the kernel's static shared memory, which the launch adds)
};
MdShape md_shape(const Sim &S);
cudaError_t launch_gather(const Sim &S, const void *A, cudaStream_t st);
// the step's starting Verlet lists, for the particle kernel that follows
cudaError_t launch_lists(const Sim &S, cudaStream_t st);
cudaError_t launch_bead_diag(const Sim &S, cudaStream_t st);
cudaError_t launch_particles(const Sim &S, const void *A, cudaStream_t st);
// clusters of the particle kernel's shape for S that can be resident at once
cudaError_t particles_clusters_fit(const Sim &S, int *n_fit);
cudaError_t launch_bead_observables(const Sim &S, const void *A, cudaStream_t st);
// reverse mode (FP32 populations only)
cudaError_t launch_sc_adjoint(const Sim &S, const void *A, const float *Lin, float *Lout, int by, int zc, cudaStream_t st);
size_t bead_adjoint_smem(const Sim &S);
cudaError_t launch_bead_adjoint(const Sim &S, const void *A, const float *Lin, const float4 *trj, float4 *lam_r, float4 *lam_v,
                                unsigned long long *LU, int *adj_node, double *dpar, long long step, cudaStream_t st);
cudaError_t launch_adj_fixup(const Sim &S, const void *A, float *Lout, const int *adj_node, unsigned long long *LU, int *stamp,
                             int tag, cudaStream_t st);

}  // namespace lbmd
