// k_particles.cu -- bead side of the coupled LB-MD step:
//   1. gather kernel (one warp per bead across the GPU, 4 lanes per corner):
//      fluid velocity at every bead from the populations the step starts from
//      (trilinear over fluid corners), frozen for the MD cycle (Sec. II, text
//      after Eq. 21), plus the corner sites and weights the spread reuses;
//   2. particle kernel: the MD cycle (Sec. II, Eq. 22 as multiple-time-step
//      velocity Verlet): M outer steps whose half kicks apply the pore field,
//      the friction gamma (u_p - v) and Philox noise (Eqs. 12, 13, 15), around
//      M^b velocity-Verlet sub-steps of the conservative forces (harmonic bonds
//      Eq. 19, angular term, WCA between beads Eq. 14 and with solid sites),
//      accumulating the momentum J the fluid handed over; then the spread
//      G(x) -= W(x - r_p) J_p with the gather's weights, as 2^40 fixed-point
//      integer atomics (order-independent, so runs repeat bit for bit).
//
// Layout of the particle kernel.  A chain takes ceil(N / Nc) consecutive
// blocks of one thread-block cluster of C blocks; short chains share a
// cluster.  Block c owns Nc consecutive beads, and each bead is worked on by
// T consecutive threads that split its pair and wall terms and add them with
// a butterfly of shuffles.  The bonded terms (bonds, the three angles that
// involve a bead) are either split over the same T lanes, or, in the
// bonded-warp kernels (BWM), evaluated once per bond and angle by extra warps
// at the end of the block (see bonded_stage).  Every block keeps a
// replica of the chain's positions in shared memory, exchanged through
// distributed shared memory in one of two ways (S.md_pull, chosen by the
// autotuner): push, where a bead's new position is written to every replica
// of its chain before the cluster barrier of each sub-step; or pull, where it
// goes into its own block's replica only, and after the barrier each block
// copies its halo (the other blocks' beads that its bonds, angles and pair
// lists read) from their owners, and a list rebuild copies the whole chain.
// Push costs each block a store per bead and replica, pull one round trip per
// sub-step for a few beads.  Bead-bead pairs come from a
// Verlet list (cut-off + skin), built by a scan of the whole chain by all
// lanes (chains up to 512 beads) or from a cell hash in shared memory, and
// rebuilt whenever any bead has moved more than half the skin since the last
// build, so the pair set equals all pairs inside the cut-off at every
// evaluation.  The bead diagnostics of the step are summed by their own
// kernel, beside this one, from the starting state the gather saves.
#include <cooperative_groups.h>

#include "lbmd_internal.cuh"

namespace cg = cooperative_groups;

namespace lbmd {

__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
// a - b for two unwrapped float-float positions (bonded neighbours: no minimum image)
__device__ __forceinline__ float3 ffsub(float4 ah, float4 al, float4 bh, float4 bl) {
    return make_float3((ah.x - bh.x) + (al.x - bl.x), (ah.y - bh.y) + (al.y - bl.y), (ah.z - bh.z) + (al.z - bl.z));
}

// ---------------------------------------------------------------------------
// lattice corner c (0..7) of the cell holding a bead at wrapped (xw, yw, zw)
// (xw in the whole lattice): the corner's local plane xi, its local site index
// and raw trilinear weight (solid corners are zeroed by the caller from the
// site's link word).  xc0 is the cell's first plane in local coordinates.  In
// slab mode a cell that does not lie inside the local planes gives weight 0
// and site 0 (the bead is not this slab's).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void corner_of(const Sim &S, float xw, float yw, float zw, int c, int &xi, int &yi,
                                          int &zi, int &node, float &w, int &xc0) {
    const int x0 = (int)floorf(xw), y0 = (int)floorf(yw), z0 = (int)floorf(zw);
    const float fx = xw - (float)x0, fy = yw - (float)y0, fz = zw - (float)z0;
    const int a = c & 1, b = (c >> 1) & 1, d = c >> 2;
    int xl = x0 - S.gx0;
    if (xl < 0) xl += S.bnx;
    // a slab as wide as the lattice (less up to three planes) holds some
    // cells twice, as ghosts and as its own: take its own copy
    if (S.slab && xl < S.own_lo && xl + S.bnx <= S.nx - 2) xl += S.bnx;
    xc0 = xl;
    const bool here = !S.slab || xl <= S.nx - 2;
    xi = S.slab ? (here ? xl + a : 0) : wrapi(xl + a, S.nx);
    yi = wrapi(y0 + b, S.ny);
    zi = wrapi(z0 + d, S.nz);
    node = xi + S.nx * (yi + S.ny * zi);
    w = (a ? fx : 1.0f - fx) * (b ? fy : 1.0f - fy) * (d ? fz : 1.0f - fz);
    if (S.interp == 1)  // nearest grid point: the corner on the bead's side of each mid-plane
        w = (a == (fx >= 0.5f) && b == (fy >= 0.5f) && d == (fz >= 0.5f)) ? 1.0f : 0.0f;
    if (!here) w = 0.0f;
}

// Sum over the 8 corners: lane l holds corner l >> 2, and the xor tree over
// 4, 8, 16 visits the 8 lanes l ^ m that share l's sub-lane, one per corner,
// so every lane gets the full sum as long as all 4 sub-lanes of a corner hold
// the same value.
__device__ __forceinline__ float corner_sum(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    return v;
}
__device__ __forceinline__ float sub_sum(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    return v;
}

// Fluid velocity at one bead, computed by a whole warp: lanes 4c..4c+3 pull the
// 19 populations of corner c (links i with i % 4 == lane % 4), form rho and
// rho u there, and the corners are combined with the renormalised weights.
// The pulled value and its bounce-back alternative are both loaded up front,
// so every load of the warp is in flight at once (no dependent chain through
// the link word).  Each lane returns its corner's site and normalised weight.
template <typename T>
__device__ __forceinline__ float3 gather_warp(const Sim &S, const T *__restrict__ A, float xw, float yw, float zw,
                                              int &node, float &W, int &xi, int &xc0) {
    const int lane = threadIdx.x & 31, c = lane >> 2, sub = lane & 3;
    int yi, zi;
    float w;
    corner_of(S, xw, yw, zw, c, xi, yi, zi, node, w, xc0);
    const uint32_t ns = (uint32_t)S.ps;  // population stride
    const uint32_t lm = __ldg(S.link + node);
    float hp[5], hb[5];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if ((i & 3) != sub) continue;
        const uint32_t src = (uint32_t)(wrapi(xi - cx(i), S.nx) + S.nx * (wrapi(yi - cy(i), S.ny) + S.ny * wrapi(zi - cz(i), S.nz)));
        hp[i >> 2] = load_dev_cg(A, (uint32_t)i * ns + src);
        hb[i >> 2] = load_dev_cg(A, (uint32_t)opp(i) * ns + (uint32_t)node);
    }
    if (lm & SOLID_BIT) w = 0.0f;
    const float wsum = corner_sum(w);
    W = wsum > 0.0f ? w / wsum : 0.0f;
    float m = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;  // rho - 1 and rho u at the corner
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if ((i & 3) != sub) continue;
        const float h = ((lm >> i) & 1u) ? hb[i >> 2] : hp[i >> 2];
        m += h;
        jx += (float)cx(i) * h;
        jy += (float)cy(i) * h;
        jz += (float)cz(i) * h;
    }
    m = sub_sum(m); jx = sub_sum(jx); jy = sub_sum(jy); jz = sub_sum(jz);
    float ux = 0.f, uy = 0.f, uz = 0.f;
    const float rho = 1.0f + m;
    if (w > 0.0f && rho > 0.0f) { ux = w * (jx / rho); uy = w * (jy / rho); uz = w * (jz / rho); }
    ux = corner_sum(ux); uy = corner_sum(uy); uz = corner_sum(uz);
    if (wsum > 0.0f) return make_float3(ux / wsum, uy / wsum, uz / wsum);
    return make_float3(0.f, 0.f, 0.f);
}

// ---------------------------------------------------------------------------
// gather kernel: one warp per bead over the whole GPU.  Writes the frozen fluid
// velocity u_p and the (site, weight) of the bead's 8 corners, which the
// spread of the same step reuses (adjoint pair: same weights both ways).
// ---------------------------------------------------------------------------
template <int PREC>
__global__ void __launch_bounds__(256) k_gather(const Sim S, const void *__restrict__ Av) {
    using T = typename PopT<PREC>::T;
    const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;  // global bead index
    if (g >= S.total_beads) return;
    const int r = S.bead_real[g];
    const T *A = reinterpret_cast<const T *>(Av) + (size_t)r * Q * S.ps;
    const float4 qh = S.r_hi[g], ql = S.r_lo[g];
    int node, xi, xc0;
    float W;
    const float3 u = gather_warp(S, A, ff_wrap(qh.x, ql.x, (float)S.bnx, S.binx), ff_wrap(qh.y, ql.y, (float)S.ny, S.iny),
                                 ff_wrap(qh.z, ql.z, (float)S.nz, S.inz), node, W, xi, xc0);
    const int lane = threadIdx.x & 31;
    // u_p from the handle that owns the bead's cell (every handle without
    // slabs); in slab mode the others give 0 and the handles' values are summed
    const bool cell_own = xc0 >= S.own_lo && xc0 < S.own_hi;
    if (lane == 0) S.up[g] = cell_own ? make_float4(u.x, u.y, u.z, 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
    // the starting state, for the step's bead diagnostics (the particle
    // kernel overwrites r and v while the lattice pass that sums them runs)
    if (lane == 1) S.bsnap[g] = qh;
    if (lane == 2) S.bsnap[S.total_beads + g] = ql;
    if (lane == 3) S.bsnap[2 * S.total_beads + g] = S.v[g];
    if ((lane & 3) == 0) {
        // the spread reaches the corners this handle owns (a ghost corner of
        // a slab as wide as the lattice is also its own plane xi - bnx)
        const int c = lane >> 2;
        const int xs = (S.slab && xi >= S.own_hi && xi - S.bnx >= S.own_lo) ? xi - S.bnx : xi;
        const bool mine = W > 0.0f && xs >= S.own_lo && xs < S.own_hi;
        S.pair_node[(size_t)g * 8 + c] = mine ? (int)((size_t)r * S.ns + node + (xs - xi)) : -1;
        S.pair_w[(size_t)g * 8 + c] = W;
    }
}

// ---------------------------------------------------------------------------
// Bead part of the per-step diagnostics row (one block per realization), from
// the starting state the gather kernel saved; it runs beside the lattice pass
// and the particle kernel.  Every term enters as 64-bit fixed point
// (fix_of): exact sums, in any order.
// ---------------------------------------------------------------------------
// x - c for x = hi + lo and c = chi + clo, as a float-float pair (h, l):
// Knuth's two-sum of hi and -chi, then the low parts added to the error term
__device__ __forceinline__ void diff_ff(float hi, float lo, float chi, float clo, float &h, float &l) {
    h = hi - chi;
    const float bb = h - hi;
    l = ((hi - (h - bb)) + (-chi - bb)) + (lo - clo);
}

// One pass over the realization's beads, adding its terms into sb:
//   PASS 0: momentum, translocated count, work rates   -> sb 0, 1, 2, 6, 7, 8
//   PASS 1: positions of all beads and of the translocated ones -> 3-5, 9-11
//   PASS 2: |r - c|^2 about each part's centroid c (in cen)     -> 12, 13
template <int PASS>
__device__ __forceinline__ void bead_sum_pass(const Sim &S, int off, int N, unsigned long long *sb, const float *cen) {
    constexpr int NV = PASS == 2 ? 2 : 6;
    const int TB = S.total_beads;
    const float thr = (float)S.wall_x + 0.5f;
    long long a[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) a[k] = 0;
    const int trips = (N + blockDim.x - 1) / blockDim.x;  // uniform over the block
    for (int it = 0; it < trips; ++it) {
        const int q = it * blockDim.x + threadIdx.x;
        if (q >= N) continue;
        const float4 h = S.bsnap[off + q], l = S.bsnap[TB + off + q];
        // x = hi + lo > thr, exactly: a stored position is normalised
        // (|lo| <= ulp(hi) / 2), so hi decides unless it equals thr
        const bool tr = S.wall_x >= 0 && (h.x > thr || (h.x == thr && l.x > 0.0f));
        if constexpr (PASS == 0) {
            const float4 v = S.bsnap[2 * TB + off + q], u = S.up[off + q];
            const bool ch = in_channel(S, ff_wrap(h.x, l.x, (float)S.bnx, S.binx), ff_wrap(h.y, l.y, (float)S.ny, S.iny),
                                       ff_wrap(h.z, l.z, (float)S.nz, S.inz));
            a[0] += fix_of(v.x, FIXD_V); a[1] += fix_of(v.y, FIXD_V); a[2] += fix_of(v.z, FIXD_V);
            a[3] += tr ? 1 : 0;
            a[4] += fix_of(S.gamma * fmaf(v.x, u.x, fmaf(v.y, u.y, v.z * u.z)), FIXD_V);
            a[5] += ch ? fix_of(S.E * v.x, FIXD_V) : 0;
        } else if constexpr (PASS == 1) {
            const long long X = fix_of(h.x, FIXD_X) + fix_of(l.x, FIXD_X);
            const long long Y = fix_of(h.y, FIXD_X) + fix_of(l.y, FIXD_X);
            const long long Z = fix_of(h.z, FIXD_X) + fix_of(l.z, FIXD_X);
            a[0] += X; a[1] += Y; a[2] += Z;
            a[3] += tr ? X : 0; a[4] += tr ? Y : 0; a[5] += tr ? Z : 0;
        } else {
            const float *c = cen + (tr ? 6 : 0);  // (hi, lo) per axis of this bead's part
            const float hc[3] = {h.x, h.y, h.z}, lc[3] = {l.x, l.y, l.z};
            long long d2 = 0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                float dh, dl;
                diff_ff(hc[k], lc[k], c[2 * k], c[2 * k + 1], dh, dl);
                // d^2 = p + e up to the dl^2 term, p + e from one exact product
                const float p = dh * dh;
                const float e = fmaf(2.0f * dh, dl, fmaf(dh, dh, -p));
                d2 += fix_of(p, FIXD_D2) + fix_of(e, FIXD_D2);
            }
            a[tr ? 1 : 0] += d2;
        }
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const long long w = warp_sum_ll(a[k]);
        const int dst = PASS == 0 ? (k < 3 ? k : k + 3) : (PASS == 1 ? (k < 3 ? 3 + k : 6 + k) : 12 + k);
        if ((threadIdx.x & 31) == 0 && w != 0) atomicAdd(sb + dst, (unsigned long long)w);
    }
}

// Bead momentum, centre of mass, translocated count (x > wall_x + 1/2,
// unwrapped), the work rates gamma v.u_p and F_E.v (Sec. IV.C), and the radii
// of gyration of the untranslocated and translocated parts, two-pass:
// centroids from exact sums, then the squared distances to them (Sec. IV.B).
// Thread 0 writes them into the step's row and advances the realization's
// translocation record (Sec. IV.A).
__global__ void __launch_bounds__(256) k_bead_diag(const Sim S) {
    __shared__ unsigned long long sb[14];
    __shared__ float cen[12];
    const int rr = blockIdx.x, tid = threadIdx.x;
    const int off = S.bead_off[rr], N = S.bead_off[rr + 1] - off;
    const long long step = S.ctrl->step;
    if (tid < 14) sb[tid] = 0ull;
    __syncthreads();
    bead_sum_pass<0>(S, off, N, sb, cen);
    bead_sum_pass<1>(S, off, N, sb, cen);
    __syncthreads();
    const long long nTi = (long long)sb[6];
    const double nT = (double)nTi, nU = (double)(N - nTi);
    const double ux = fix_unit(FIXD_X);
    if (tid < 6) {  // centroid of the untranslocated (0..2) or translocated (3..5) part, one axis
        const int k = tid % 3;
        const bool t = tid >= 3;
        const long long all = (long long)sb[3 + k], trs = (long long)sb[9 + k];
        const double n = t ? nT : nU;
        const double c = n > 0 ? (double)(t ? trs : all - trs) * ux / n : 0.0;
        const float chi = (float)c;
        cen[(t ? 6 : 0) + 2 * k] = chi;
        cen[(t ? 6 : 0) + 2 * k + 1] = (float)(c - (double)chi);
    }
    __syncthreads();
    bead_sum_pass<2>(S, off, N, sb, cen);
    __syncthreads();
    if (tid != 0) return;
    const double uv = fix_unit(FIXD_V), ud = fix_unit(FIXD_D2);
    lbmd_diag *row = S.ring + (size_t)rr * LBMD_DIAG_RING + (step % LBMD_DIAG_RING);
    row->p_beads[0] = (double)(long long)sb[0] * uv;
    row->p_beads[1] = (double)(long long)sb[1] * uv;
    row->p_beads[2] = (double)(long long)sb[2] * uv;
    const double inv = N > 0 ? ux / N : 0.0;
    row->com[0] = (double)(long long)sb[3] * inv;
    row->com[1] = (double)(long long)sb[4] * inv;
    row->com[2] = (double)(long long)sb[5] * inv;
    row->n_translocated = nT;
    row->dWH_dt = (double)(long long)sb[7] * uv;
    row->dWE_dt = (double)(long long)sb[8] * uv;
    const double rgU = nU > 0 ? sqrt((double)(long long)sb[12] * ud / nU) : 0.0;
    const double rgT = nT > 0 ? sqrt((double)(long long)sb[13] * ud / nT) : 0.0;
    row->rg_untranslocated = rgU;
    row->rg_translocated = rgT;
    lbmd_transloc *ev = S.tl + rr;
    if (N > 0 && step >= ev->t_origin) {
        if (step == ev->t_origin) ev->rg_u_origin = rgU;
        if (nT > ev->max_translocated) ev->max_translocated = nT;
        if (ev->t_first < 0 && nTi > 0) ev->t_first = step;
        if (ev->t_x < 0 && nTi >= N) { ev->t_x = step; ev->rg_t_x = rgT; }
    }
}

cudaError_t launch_bead_diag(const Sim &S, cudaStream_t st) {
    if (S.total_beads == 0) return cudaSuccess;
    k_bead_diag<<<S.n_real, 256, 0, st>>>(S);
    return cudaGetLastError();
}

cudaError_t launch_gather(const Sim &S, const void *A, cudaStream_t st) {
    if (S.total_beads == 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (S.total_beads * 32 + threads - 1) / threads;
    if (S.precision == LBMD_FP16DEV) k_gather<1><<<blocks, threads, 0, st>>>(S, A);
    else k_gather<0><<<blocks, threads, 0, st>>>(S, A);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// conservative (fast) force terms
// ---------------------------------------------------------------------------
// angle between b1 and b2 (phi = atan2(|b1 x b2|, b1.b2)), V = kappa phi^2 / 2:
// d1 = A dcos/db1, d2 = A dcos/db2 with A = kappa phi / sin(phi)
__device__ __forceinline__ void bend_terms(float3 b1, float3 b2, float kappa, float3 &d1, float3 &d2) {
    const float l1s = dot3(b1, b1), l2s = dot3(b2, b2), dt = dot3(b1, b2);
    const float3 cr = cross3(b1, b2);
    const float cr2 = dot3(cr, cr);
    const float crn = cr2 > 0.0f ? cr2 * rsqrtf(cr2) : 0.0f;
    const float inv12 = rsqrtf(l1s * l2s);
    const float c = dt * inv12, sn = crn * inv12;
    const float phi = atan_pos(crn, dt);
    const float A = sn > 1e-6f ? __fdividef(kappa * phi, sn) : (c > 0.0f ? kappa : 0.0f);
    d1 = A * (inv12 * b2 - __fdividef(c, l1s) * b1);
    d2 = A * (inv12 * b1 - __fdividef(c, l2s) * b2);
}

// WCA (Eq. 14 cut at its minimum, shifted): -dV/dd = coef * d.  1/r^2 from
// the hardware reciprocal (within about an ulp; the pair terms sit on the
// sub-step's dependent chain, where the correctly rounded one costs a
// Newton refinement)
__device__ __forceinline__ float wca_coef(float r2, float eps, float sig2) {
    const float ir2 = __fdividef(1.0f, r2), sr2 = sig2 * ir2;
    const float sr6 = sr2 * sr2 * sr2;
    return 24.0f * eps * (2.0f * sr6 * sr6 - sr6) * ir2;
}

struct PSmem {
    // replica of the whole chain: positions hi / lo, double buffered.  Two
    // members behind a select, not an array indexed by the buffer number: a
    // runtime index into the struct would keep it in local memory, and every
    // sub-step would load these pointers from there
    float4 *ph0, *ph1, *pl0, *pl1;
    __device__ __forceinline__ float4 *ph(int b) const { return b ? ph1 : ph0; }
    __device__ __forceinline__ float4 *pl(int b) const { return b ? pl1 : pl0; }
    float4 *jbuf;           // [Nc] impulse J of the block's beads, for the spread
    uint16_t *nbr;          // [Nc][NBR_CAP] bead-pair lists of the block's beads
    uint32_t *wal;          // [Nc][WALL_CAP] packed solid-site coordinates
    int *hkey, *hhead;      // [HASH_SIZE] cell hash
    int16_t *hnext;         // [Nmax] cell lists
    uint8_t *nn, *nw;       // [Nc] list lengths
    float4 *znz;            // [Nc][Mb] noise of the SPV inner steps of one outer step (or none)
    uint32_t *halo;         // [Nmax] the other blocks' beads this block's force terms read: q | owner rank << 16
    uint8_t *mark;          // [Nmax] scratch of the halo build
    float4 *bnd;            // [Nc + 2][3] bonded terms of the centres first-1 .. last+1 (bonded_stage)
};

// nzn: float4 slots for the SPV noise (Nc * Mb when that cycle draws noise, else 0)
// warps of the bonded terms for blocks of nc beads: one lane per centre
__host__ __device__ inline int bonded_warps(int nc) { return (nc + 2 + 31) / 32; }

__host__ __device__ inline size_t psmem_layout(int nmax, int nc, int nzn, PSmem *p, char *base) {
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o += (bytes + 15) & ~(size_t)15; return base + at; };
    char *ph0 = take(16 * (size_t)nmax), *ph1 = take(16 * (size_t)nmax);
    char *pl0 = take(16 * (size_t)nmax), *pl1 = take(16 * (size_t)nmax);
    char *jb = take(16 * (size_t)nc);
    char *nbr = take(2 * (size_t)NBR_CAP * nc);
    char *wal = take(4 * (size_t)WALL_CAP * nc);
    char *hkey = take(4 * (size_t)HASH_SIZE), *hhead = take(4 * (size_t)HASH_SIZE);
    char *hnext = take(2 * (size_t)nmax);
    char *nn = take((size_t)nc), *nw = take((size_t)nc);
    char *znz = take(16 * (size_t)nzn);
    char *halo = take(4 * (size_t)nmax), *mark = take((size_t)nmax);
    char *bnd = take(48 * ((size_t)nc + 2));
    if (p) {
        p->ph0 = (float4 *)ph0; p->ph1 = (float4 *)ph1;
        p->pl0 = (float4 *)pl0; p->pl1 = (float4 *)pl1;
        p->jbuf = (float4 *)jb;
        p->nbr = (uint16_t *)nbr; p->wal = (uint32_t *)wal;
        p->hkey = (int *)hkey; p->hhead = (int *)hhead; p->hnext = (int16_t *)hnext;
        p->nn = (uint8_t *)nn; p->nw = (uint8_t *)nw;
        p->znz = (float4 *)znz;
        p->halo = (uint32_t *)halo;
        p->mark = (uint8_t *)mark;
        p->bnd = (float4 *)bnd;
    }
    return o;
}

// noise slots of the SPV cycle: one float4 per bead of a block and inner step
__host__ __device__ inline int spv_noise_slots(const Sim &S, int nc) {
    return (S.integrator == 1 && S.spv_sig > 0.0f) ? nc * S.Mb : 0;
}

// Automatic shape: 4 lanes per bead.  A single chain is spread over up to 8
// blocks (about 50 beads per block: the sub-step is latency-bound, so fewer
// beads per SM shorten it); an ensemble keeps each chain in as few blocks as
// fit (<= 512 threads per block), since its realizations already fill the
// GPU.  A shape set through lbmd_set_md_shape (S.md_T, S.md_C) takes
// precedence.
MdShape md_shape(const Sim &S) {
    MdShape m;
    const int N = S.max_beads;
    m.T = S.md_T > 0 ? S.md_T : 4;
    const int per_block = 512 / m.T;
    const int fit = max(1, (N + per_block - 1) / per_block);
    const int spread = S.n_real == 1 ? min(8, max(fit, (N + 49) / 50)) : fit;
    m.C = S.md_C > 0 ? S.md_C : spread;
    m.Nc = N > 0 ? (N + m.C - 1) / m.C : 1;
    // the bonded warp: by request, else for blocks of at most 30 beads
    m.bw = S.md_bw == 2 || (S.md_bw == 0 && m.Nc + 2 <= 32);
    m.threads = max(32, ((m.Nc * m.T + 31) / 32) * 32) + (m.bw ? 32 * bonded_warps(m.Nc) : 0);
    m.smem = psmem_layout(max(N, 1), m.Nc, spv_noise_slots(S, m.Nc), nullptr, nullptr);
    // Reserving: a block launched with the device's whole opt-in shared
    // memory leaves its SM too little for any block of the other kernels, so
    // the lattice pass and the gather do not share the particle kernel's SMs.
    // The launch trims this by the kernel's static shared memory.
    m.launch_smem = S.md_reserve ? max(m.smem, (size_t)max(S.smem_optin, 0)) : m.smem;
    return m;
}

// Part of the conservative force on bead p computed by task lane lt of its
// T lanes.  Terms: harmonic bonds (Eq. 19); the angular term of the angles at
// p-1, p, p+1; WCA with the listed beads and solid sites.  The lanes' parts
// add up to the full force.  Every lane of the warp must call this (own or
// not): the list loops run to a warp-uniform trip count.
// bonded_part: the bond and angle terms, which read beads p-2 .. p+2 only;
// pair_part: adds the pair- and wall-list terms to them.  force_part is both.
template <int T>
__device__ __forceinline__ float3 bonded_part(const Sim &S, const PSmem &sm, int buf, bool own, int p, int N, float4 mh,
                                              float4 ml, int lt) {
    float3 F = make_float3(0.f, 0.f, 0.f);
    const float4 *ph = sm.ph(buf), *plo = sm.pl(buf);
    if constexpr (T >= 3) {
        // Lane lt (< 3) takes the angle whose beads are a = p+lt-2,
        // b = p+lt-1, c = p+lt, with u = r_b - r_a and w = r_c - r_b.  Its
        // share of the force on p (p = c, b, a for lt = 0, 1, 2) is
        // +A dcos/dw, A (dcos/du - dcos/dw), -A dcos/du.  Lanes 0 and 1 also
        // take the bond along w (p = c: -k(|w| - r0) w/|w|; p = b: +...).
        // Straight-line code with selects, for every lane (own or not: a
        // lane without a bead reads bead 0 and selects nothing), so that the
        // bond and angle chains and the pair terms that follow share one
        // basic block and overlap.
        {
            const int pb = own ? p : 0;
            const int ia = pb + lt - 2, ib = pb + lt - 1, ic = pb + lt;
            const bool va = own && ia >= 0 && ia < N, vb = own && ib >= 0 && ib < N, vc = own && ic >= 0 && ic < N;
            const int ja = va ? ia : pb, jb = vb ? ib : pb, jc = vc ? ic : pb;
            const float4 ha = ph[ja], la = plo[ja], hb = ph[jb], lb = plo[jb], hc = ph[jc], lc = plo[jc];
            const float3 u = ffsub(hb, lb, ha, la), w = ffsub(hc, lc, hb, lb);
            const bool bond_ok = lt < 2 && vb && vc;
            const bool ang_ok = lt < 3 && va && vb && vc && S.kappa != 0.0f;
            // |w| from the correctly rounded sqrt: |w| - r0 cancels and keeps
            // only the absolute error of |w|
            const float w2 = bond_ok ? dot3(w, w) : 1.0f;
            const float len = sqrtf(w2);
            const float bc = __fdividef(S.k_bond * (len - S.r0), len);
            const float bsign = lt == 0 ? -1.0f : 1.0f;
            const float3 uu = ang_ok ? u : make_float3(1.f, 0.f, 0.f);
            const float3 ww = ang_ok ? w : make_float3(0.f, 1.f, 0.f);
            float3 d1, d2;
            bend_terms(uu, ww, S.kappa, d1, d2);
            const float al = lt == 0 ? 0.0f : (lt == 1 ? 1.0f : -1.0f);
            const float be = lt == 0 ? 1.0f : (lt == 1 ? -1.0f : 0.0f);
            if (bond_ok) F = F + (bsign * bc) * w;
            if (ang_ok) F = F + al * d1 + be * d2;
        }
    } else if (own) {
        {
            const bool m1 = p >= 1, m2 = p >= 2, p1 = p + 1 < N, p2 = p + 2 < N;
            float4 hm1 = mh, lm1 = ml, hm2 = mh, lm2 = ml, hp1 = mh, lp1 = ml, hp2 = mh, lp2 = ml;
            if (m1) { hm1 = ph[p - 1]; lm1 = plo[p - 1]; }
            if (m2) { hm2 = ph[p - 2]; lm2 = plo[p - 2]; }
            if (p1) { hp1 = ph[p + 1]; lp1 = plo[p + 1]; }
            if (p2) { hp2 = ph[p + 2]; lp2 = plo[p + 2]; }
            const float3 b0 = ffsub(hm1, lm1, hm2, lm2);  // r_{p-1} - r_{p-2}
            const float3 b1 = ffsub(mh, ml, hm1, lm1);    // r_p - r_{p-1}
            const float3 b2 = ffsub(hp1, lp1, mh, ml);    // r_{p+1} - r_p
            const float3 b3 = ffsub(hp2, lp2, hp1, lp1);  // r_{p+2} - r_{p+1}
            // bond slots: 0 = bond to p-1, 1 = bond to p+1
            for (int s = lt; s < 2; s += T) {
                const float3 b = s == 0 ? b1 : b2;
                if (s == 0 ? m1 : p1) {
                    const float len = sqrtf(dot3(b, b));
                    const float coef = __fdividef(S.k_bond * (len - S.r0), len);
                    F = F + (s == 0 ? -coef : coef) * b;
                }
            }
            // angle slots: the angles at p-1, p, p+1
            if (S.kappa != 0.0f) {
                for (int s = lt; s < 3; s += T) {
                    const float3 u = s == 0 ? b0 : (s == 1 ? b1 : b2);
                    const float3 w = s == 0 ? b1 : (s == 1 ? b2 : b3);
                    if (s == 0 ? m2 : (s == 1 ? (m1 && p1) : p2)) {
                        float3 d1, d2;
                        bend_terms(u, w, S.kappa, d1, d2);
                        const float al = s == 0 ? 0.0f : (s == 1 ? 1.0f : -1.0f);
                        const float be = s == 0 ? 1.0f : (s == 1 ? -1.0f : 0.0f);
                        F = F + al * d1 + be * d2;
                    }
                }
            }
        }
    }
    return F;
}

// Bonded warps (by default for blocks of at most 30 beads, one warp): each
// bond and angle is evaluated once per block by the block's last
// ceil((Nc + 2) / 32) warps (bonded_stage), which leave their terms in
// shared memory, while the other warps sum the pair and wall terms with T
// lanes per bead (pair_part); full_force adds the two.  Without them, an
// angle is evaluated by each of its three beads' lanes and a bond by both of
// its beads' (bonded_part), which costs every warp the bonded instructions
// but needs no block barrier and no extra threads.
//
// bonded_stage: slot s of sm.bnd holds, for centre j = first - 1 + s
// (first = the block's first bead), the angle terms d1 = A dcos/du and
// d2 = A dcos/dw of u = r_j - r_{j-1}, w = r_{j+1} - r_j (zero where the angle
// does not exist or kappa = 0) and the bond term k (|w| - r0) w / |w| of
// (j, j+1) (zero where that bond does not exist).  Called by the 32 lanes of
// one warp; the block's own beads need the centres first - 1 .. last + 1.
__device__ __forceinline__ void bonded_stage(const Sim &S, const PSmem &sm, int buf, int N, int Nc, int first,
                                             int last) {
    const float4 *ph = sm.ph(buf), *plo = sm.pl(buf);
    const int nctr = last >= first ? last - first + 3 : 0;
    const int nbt = 32 * bonded_warps(Nc);  // the block's last nbt threads
    for (int sl = threadIdx.x - (blockDim.x - nbt); sl < nctr; sl += nbt) {
        const int j = first - 1 + sl;
        const bool bond_ok = j >= 0 && j + 1 < N;
        const bool ang_ok = j >= 1 && j + 1 < N && S.kappa != 0.0f;
        const int jb = min(max(j, 0), N - 1);
        const int ja = bond_ok || ang_ok ? max(j - 1, 0) : jb, jc = min(jb + 1, N - 1);
        const float4 ha = ph[ja], la = plo[ja], hb = ph[jb], lb = plo[jb], hc = ph[jc], lc = plo[jc];
        const float3 u = ffsub(hb, lb, ha, la), w = ffsub(hc, lc, hb, lb);
        // |w| from the correctly rounded sqrt: |w| - r0 cancels and keeps
        // only the absolute error of |w|
        const float w2 = bond_ok ? dot3(w, w) : 1.0f;
        const float len = sqrtf(w2);
        const float bc = __fdividef(S.k_bond * (len - S.r0), len);
        const float3 uu = ang_ok ? u : make_float3(1.f, 0.f, 0.f);
        const float3 ww = ang_ok ? w : make_float3(0.f, 1.f, 0.f);
        float3 d1, d2;
        bend_terms(uu, ww, S.kappa, d1, d2);
        const float3 z = make_float3(0.f, 0.f, 0.f);
        if (!ang_ok) { d1 = z; d2 = z; }
        const float3 bw = bond_ok ? bc * w : z;
        sm.bnd[3 * sl + 0] = make_float4(d1.x, d1.y, d1.z, 0.f);
        sm.bnd[3 * sl + 1] = make_float4(d2.x, d2.y, d2.z, 0.f);
        sm.bnd[3 * sl + 2] = make_float4(bw.x, bw.y, bw.z, 0.f);
    }
}

// Bonded force on the bead of slot s (s = p - first + 1) from the terms of
// the slots s - 1, s, s + 1, in a fixed order: the bonds to p-1 and p+1, then
// the angles centred at p-1 (p is its c), p (its b) and p+1 (its a).
__device__ __forceinline__ float3 bonded_of(const PSmem &sm, int s) {
    const float4 b0 = sm.bnd[3 * (s - 1) + 2], b1 = sm.bnd[3 * s + 2];
    const float4 d2m = sm.bnd[3 * (s - 1) + 1], d1c = sm.bnd[3 * s + 0], d2c = sm.bnd[3 * s + 1];
    const float4 d1p = sm.bnd[3 * (s + 1) + 0];
    float3 F = make_float3(b1.x - b0.x, b1.y - b0.y, b1.z - b0.z);
    F = F + make_float3(d2m.x, d2m.y, d2m.z);
    F = F + make_float3(d1c.x - d2c.x, d1c.y - d2c.y, d1c.z - d2c.z);
    F = F - make_float3(d1p.x, d1p.y, d1p.z);
    return F;
}

template <int T>
__device__ __forceinline__ float3 pair_part(const Sim &S, const PSmem &sm, int buf, bool own, int p, int pl, float4 mh,
                                            float4 ml, int lt, float3 F) {
    const float4 *ph = sm.ph(buf), *plo = sm.pl(buf);
    const int nn = own ? (int)sm.nn[pl] : 0, nw = own ? (int)sm.nw[pl] : 0;
    const int nn_w = __reduce_max_sync(0xffffffffu, nn), nw_w = __reduce_max_sync(0xffffffffu, nw);
    const float fnx = (float)S.bnx, fny = (float)S.ny, fnz = (float)S.nz;
    // Pair and wall lists, two entries per iteration, to the warp's longest
    // list: both entries' shared-memory loads are issued before either is
    // used, and no lane branches away (entries past a lane's own list point
    // at the bead itself and are selected out).  The first pair iteration
    // runs unconditionally, in the basic block of the bonded terms, so that
    // its chain overlaps theirs (with no entries it adds zeros).
    {
        const uint16_t *lst = sm.nbr + (own ? pl : 0) * NBR_CAP;
        const int pself = own ? p : 0;  // a bead of the replica for lanes without one
        for (int k = lt; k == lt || k < nn_w; k += 2 * T) {
            const bool v0 = k < nn, v1 = k + T < nn;
            const int q0 = v0 ? (int)lst[k] : pself;
            const int q1 = v1 ? (int)lst[k + T] : pself;
            const float4 h0 = ph[q0], l0 = plo[q0], h1 = ph[q1], l1 = plo[q1];
            const float3 d0 = make_float3(ff_diff(mh.x, ml.x, h0.x, l0.x, fnx, S.binx), ff_diff(mh.y, ml.y, h0.y, l0.y, fny, S.iny),
                                          ff_diff(mh.z, ml.z, h0.z, l0.z, fnz, S.inz));
            const float3 d1 = make_float3(ff_diff(mh.x, ml.x, h1.x, l1.x, fnx, S.binx), ff_diff(mh.y, ml.y, h1.y, l1.y, fny, S.iny),
                                          ff_diff(mh.z, ml.z, h1.z, l1.z, fnz, S.inz));
            const float r20 = v0 ? dot3(d0, d0) : 1e30f, r21 = v1 ? dot3(d1, d1) : 1e30f;
            const float c0 = r20 < S.lj_rc2 ? wca_coef(r20, S.lj_eps, S.lj_sig2) : 0.0f;
            const float c1 = r21 < S.lj_rc2 ? wca_coef(r21, S.lj_eps, S.lj_sig2) : 0.0f;
            F = F + c0 * d0 + c1 * d1;
        }
    }
    {
        const uint32_t *wl = sm.wal + (own ? pl : 0) * WALL_CAP;
        for (int k = lt; k < nw_w; k += 2 * T) {
            const bool v0 = k < nw, v1 = k + T < nw;
            const uint32_t p0 = v0 ? wl[k] : 0u;
            const uint32_t p1 = v1 ? wl[k + T] : 0u;
            const float3 d0 = make_float3(ff_diff(mh.x, ml.x, (float)(p0 & 0xfffu), 0.f, fnx, S.binx),
                                          ff_diff(mh.y, ml.y, (float)((p0 >> 12) & 0x3ffu), 0.f, fny, S.iny),
                                          ff_diff(mh.z, ml.z, (float)(p0 >> 22), 0.f, fnz, S.inz));
            const float3 d1 = make_float3(ff_diff(mh.x, ml.x, (float)(p1 & 0xfffu), 0.f, fnx, S.binx),
                                          ff_diff(mh.y, ml.y, (float)((p1 >> 12) & 0x3ffu), 0.f, fny, S.iny),
                                          ff_diff(mh.z, ml.z, (float)(p1 >> 22), 0.f, fnz, S.inz));
            const float r20 = v0 ? dot3(d0, d0) : 1e30f, r21 = v1 ? dot3(d1, d1) : 1e30f;
            const float c0 = r20 < S.wall_rc2 ? wca_coef(r20, S.wall_eps, S.wall_sig2) : 0.0f;
            const float c1 = r21 < S.wall_rc2 ? wca_coef(r21, S.wall_eps, S.wall_sig2) : 0.0f;
            F = F + c0 * d0 + c1 * d1;
        }
    }
    if (!own) F = make_float3(0.f, 0.f, 0.f);
    return F;
}


template <int T>
__device__ __forceinline__ float3 force_part(const Sim &S, const PSmem &sm, int buf, bool own, int p, int pl, int N, float4 mh,
                                             float4 ml, int lt) {
    return pair_part<T>(S, sm, buf, own, p, pl, mh, ml, lt, bonded_part<T>(S, sm, buf, own, p, N, mh, ml, lt));
}

// sum over the T consecutive lanes of a bead (fixed butterfly: deterministic)
template <int T>
__device__ __forceinline__ float3 group_sum(float3 F) {
#pragma unroll
    for (int o = 1; o < T; o <<= 1) {
        F.x += __shfl_xor_sync(0xffffffffu, F.x, o);
        F.y += __shfl_xor_sync(0xffffffffu, F.y, o);
        F.z += __shfl_xor_sync(0xffffffffu, F.z, o);
    }
    return F;
}

// The whole conservative force on this lane's bead (zero for a lane without
// one), from replica buf; called by every thread of the block.  With a
// bonded warp (BWM) the last warp (bw) evaluates the bonded
// terms and the others the pair and wall terms, and a block barrier joins
// them; otherwise every bead's T lanes evaluate all its terms (force_part).
template <int T, bool BWM>
__device__ __forceinline__ float3 full_force(const Sim &S, const PSmem &sm, int buf, bool own, bool bw, int p, int pl,
                                             int N, int Nc, int first, int last, float4 mh, float4 ml, int lt) {
    float3 F = make_float3(0.f, 0.f, 0.f);
    if constexpr (!BWM) {
        F = group_sum<T>(force_part<T>(S, sm, buf, own, p, pl, N, mh, ml, lt));
        return own ? F : make_float3(0.f, 0.f, 0.f);
    }
    if (bw) bonded_stage(S, sm, buf, N, Nc, first, last);
    else F = group_sum<T>(pair_part<T>(S, sm, buf, own, p, pl, mh, ml, lt, F));
    __syncthreads();
    if (own) F = F + bonded_of(sm, p - first + 1);
    return F;
}

// ---------------------------------------------------------------------------
// Verlet lists: cell hash (cells >= list radius, >= 3 per axis) or all pairs
// ---------------------------------------------------------------------------
__device__ __forceinline__ int cell_slot(int key) { return (int)(((uint32_t)key * 2654435761u) >> 21); }

__device__ __forceinline__ void list_insert(uint16_t *lst, int &n, int q) {
    int pos = n;
    while (pos > 0 && lst[pos - 1] > q) {
        if (pos < NBR_CAP) lst[pos] = lst[pos - 1];
        --pos;
    }
    if (pos < NBR_CAP) lst[pos] = (uint16_t)q;
    ++n;
}

// |d|^2 < r2 with every product and sum rounded on its own (no fused
// multiply-add), so that each list build decides a pair the same way
__device__ __forceinline__ bool within2(float dx, float dy, float dz, float r2) {
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)) < r2;
}

// Solid sites within the wall-list radius of a bead at wrapped (xw, yw, zw),
// packed as x | y << 12 | z << 22 into wal (at most WALL_CAP of them, in the
// order of the 4x4x4 box's bits); returns how many there are.
__device__ __forceinline__ int wall_list(const Sim &S, float xw, float yw, float zw, uint32_t *wal) {
    int m = 0;
    const int cx0 = (int)floorf(xw), cy0 = (int)floorf(yw), cz0 = (int)floorf(zw);
    if (S.rlw < 2.0f) {
        // every site within rlw < 2 of the bead lies in the 4x4x4 box starting
        // one site below its cell corner; its solid sites are one bit mask
        unsigned long long mm = __ldg(S.bwallmask + cx0 + S.bnx * (cy0 + S.ny * cz0));
        while (mm) {
            const int bit = __ffsll((long long)mm) - 1;
            mm &= mm - 1;
            const int X = cx0 + (bit & 3) - 1, Y = cy0 + ((bit >> 2) & 3) - 1, Z = cz0 + (bit >> 4) - 1;
            if (!within2(xw - (float)X, yw - (float)Y, zw - (float)Z, S.rlw2)) continue;
            const int xx = wrapi(X, S.bnx), yy = wrapi(Y, S.ny), zz = wrapi(Z, S.nz);
            if (m < WALL_CAP) wal[m] = (uint32_t)xx | ((uint32_t)yy << 12) | ((uint32_t)zz << 22);
            ++m;
        }
    } else if (__ldg(S.blink + cx0 + S.bnx * (cy0 + S.ny * cz0)) & NEAR_SOLID_BIT) {
        const int x0 = (int)floorf(xw - S.rlw), x1 = (int)floorf(xw + S.rlw);
        const int y0 = (int)floorf(yw - S.rlw), y1 = (int)floorf(yw + S.rlw);
        const int z0 = (int)floorf(zw - S.rlw), z1 = (int)floorf(zw + S.rlw);
        for (int Z = z0; Z <= z1; ++Z)
            for (int Y = y0; Y <= y1; ++Y)
                for (int X = x0; X <= x1; ++X) {
                    const int xx = wrap_any(X, S.bnx), yy = wrap_any(Y, S.ny), zz = wrap_any(Z, S.nz);
                    if (!(__ldg(S.blink + xx + S.bnx * (yy + S.ny * zz)) & SOLID_BIT)) continue;
                    if (!within2(xw - (float)X, yw - (float)Y, zw - (float)Z, S.rlw2)) continue;
                    if (m < WALL_CAP) wal[m] = (uint32_t)xx | ((uint32_t)yy << 12) | ((uint32_t)zz << 22);
                    ++m;
                }
    }
    return m;
}

__device__ __forceinline__ void cell_of(const Sim &S, float xw, float yw, float zw, int &ci, int &cj, int &ck) {
    ci = min((int)(xw * S.cell_per_site[0]), S.ncell[0] - 1);
    cj = min((int)(yw * S.cell_per_site[1]), S.ncell[1] - 1);
    ck = min((int)(zw * S.cell_per_site[2]), S.ncell[2] - 1);
}

// Rebuild the lists of the block's beads from the block's replica (buffer
// buf), which must hold the whole chain.  Called by every thread of the block;
// clear_flag (if not null) is reset once every thread has read it.  With
// halo set (pull exchange, chain over more than one block) it also lists the
// block's halo: the beads of other blocks (rank != this block's) in its beads'
// pair lists or within two bonds of them, in no particular order, each with
// the chain rank of its block in bits 16 and up, their count in *nhalo.
// Pair list of bead p by its T lanes over every bead of the chain in
// ascending order: lane lt tests q = kT + lt and a ballot over the bead's
// lanes compacts the hits, so the list comes out sorted (the order the
// hashed build reaches by insertion) with no hash and no sort.  Every lane of
// the warp runs the same trip count: no divergence.
template <int T>
__device__ __forceinline__ int scan_pairs(const Sim &S, const float4 *ph, const float4 *plo, int N, int p, bool own,
                                          uint16_t *lst) {
    const float fnx = (float)S.bnx, fny = (float)S.ny, fnz = (float)S.nz;
    const int lane = threadIdx.x & 31, lt = lane & (T - 1);
    const int pself = own ? p : 0;
    const float4 mh = ph[pself], ml = plo[pself];
    const unsigned gshift = (unsigned)(lane - lt);
    const unsigned gmask = T == 32 ? 0xffffffffu : ((1u << T) - 1u);
    const unsigned below = (1u << lt) - 1u;
    int n = 0;
    for (int base = 0; base < N; base += T) {
        const int q = base + lt;
        const int qq = q < N ? q : pself;
        const float4 qh = ph[qq], ql = plo[qq];
        const float dx = ff_diff(mh.x, ml.x, qh.x, ql.x, fnx, S.binx), dy = ff_diff(mh.y, ml.y, qh.y, ql.y, fny, S.iny),
                    dz = ff_diff(mh.z, ml.z, qh.z, ql.z, fnz, S.inz);
        const bool hit = own && q < N && (q < p - 1 || q > p + 1) && within2(dx, dy, dz, S.rl2);
        const unsigned g = (__ballot_sync(0xffffffffu, hit) >> gshift) & gmask;
        if (hit) {
            const int pos = n + __popc(g & below);
            if (pos < NBR_CAP) lst[pos] = (uint16_t)q;
        }
        n += __popc(g);
    }
    return n;
}

// The block's halo for the pull exchange, from the lists of its beads in
// shared memory: the beads of other blocks (rank != this block's) in its
// beads' pair lists or within two bonds of them, in no particular order, each
// with the chain rank of its block in bits 16 and up, their count in *nhalo.
// Called by every thread of the block; ends with a block barrier.
template <int T>
__device__ __forceinline__ void build_halo(const PSmem &sm, int N, int p, int pl, bool own, int rank, int Nc,
                                           int *nhalo) {
    for (int q = threadIdx.x; q < N; q += blockDim.x) sm.mark[q] = 0;
    if (threadIdx.x == 0) *nhalo = 0;
    __syncthreads();
    if (own) {
        const int lt = threadIdx.x % T;
        const uint16_t *lst = sm.nbr + pl * NBR_CAP;
        const int n = sm.nn[pl];
        for (int k = lt; k < n; k += T) {
            const int q = lst[k];
            if (q / Nc != rank) sm.mark[q] = 1;
        }
        if (lt == 0)
            for (int d = -2; d <= 2; ++d) {
                const int q = p + d;
                if (q >= 0 && q < N && q / Nc != rank) sm.mark[q] = 1;
            }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < N; q += blockDim.x)
        if (sm.mark[q]) sm.halo[atomicAdd(nhalo, 1)] = (uint32_t)q | ((uint32_t)(q / Nc) << 16);
    __syncthreads();
}

// Bead-bead and bead-wall lists of the block's beads from replica buf.
// Chains of up to BRUTE_MAX beads use scan_pairs (every lane of the block
// busy); longer ones a cell hash in shared memory, scanned by one lane per
// bead.  Both give each bead's pairs within the list radius in ascending order.
template <int T>
__device__ __forceinline__ void build_lists_body(const Sim &S, const PSmem &sm, int buf, int N, int p, int pl, bool own,
                                                 int rank, int Nc, bool halo, int *clear_flag, int *s_err, int *nhalo) {
    const bool owner = own && (threadIdx.x % T) == 0;
    const bool brute = N <= BRUTE_MAX;
    const bool hashed = !brute && S.ncell[0] >= 3 && S.ncell[1] >= 3 && S.ncell[2] >= 3;
    const float fnx = (float)S.bnx, fny = (float)S.ny, fnz = (float)S.nz;
    const float4 *ph = sm.ph(buf), *plo = sm.pl(buf);
    if (hashed)
        for (int k = threadIdx.x; k < HASH_SIZE; k += blockDim.x) { sm.hkey[k] = -1; sm.hhead[k] = -1; }
    __syncthreads();
    if (clear_flag && threadIdx.x == 0) *clear_flag = 0;
    if (hashed) {
        for (int q = threadIdx.x; q < N; q += blockDim.x) {
            const float4 qh = ph[q], ql = plo[q];
            int ci, cj, ck;
            cell_of(S, ff_wrap(qh.x, ql.x, fnx, S.binx), ff_wrap(qh.y, ql.y, fny, S.iny), ff_wrap(qh.z, ql.z, fnz, S.inz),
                    ci, cj, ck);
            const int key = ci + S.ncell[0] * (cj + S.ncell[1] * ck);
            int slot = cell_slot(key);
            for (int probe = 0; probe < HASH_SIZE; ++probe) {
                const int prev = atomicCAS(sm.hkey + slot, -1, key);
                if (prev == -1 || prev == key) break;
                slot = (slot + 1) & (HASH_SIZE - 1);
            }
            sm.hnext[q] = (int16_t)atomicExch(sm.hhead + slot, q);
        }
    }
    __syncthreads();
    int n_scan = 0;
    if (brute) n_scan = scan_pairs<T>(S, ph, plo, N, p, own, sm.nbr + (own ? pl : 0) * NBR_CAP);
    if (owner) {
        const float4 mh = ph[p], ml = plo[p];
        const float xw = ff_wrap(mh.x, ml.x, fnx, S.binx), yw = ff_wrap(mh.y, ml.y, fny, S.iny),
                    zw = ff_wrap(mh.z, ml.z, fnz, S.inz);
        uint16_t *lst = sm.nbr + pl * NBR_CAP;
        int n = n_scan;
        auto consider = [&](int q) {
            if (q == p || q == p - 1 || q == p + 1) return;
            const float4 qh = ph[q], ql = plo[q];
            const float dx = ff_diff(mh.x, ml.x, qh.x, ql.x, fnx, S.binx), dy = ff_diff(mh.y, ml.y, qh.y, ql.y, fny, S.iny),
                        dz = ff_diff(mh.z, ml.z, qh.z, ql.z, fnz, S.inz);
            if (within2(dx, dy, dz, S.rl2)) list_insert(lst, n, q);
        };
        if (brute) {
            // done by scan_pairs
        } else if (hashed) {
            int ci, cj, ck;
            cell_of(S, xw, yw, zw, ci, cj, ck);
            for (int dk = -1; dk <= 1; ++dk)
                for (int dj = -1; dj <= 1; ++dj)
                    for (int di = -1; di <= 1; ++di) {
                        const int key = wrapi(ci + di, S.ncell[0]) +
                                        S.ncell[0] * (wrapi(cj + dj, S.ncell[1]) + S.ncell[1] * wrapi(ck + dk, S.ncell[2]));
                        int slot = cell_slot(key);
                        for (int probe = 0; probe < HASH_SIZE; ++probe) {
                            const int kk = sm.hkey[slot];
                            if (kk == key) {
                                for (int q = sm.hhead[slot], guard = 0; q >= 0 && guard < N; q = sm.hnext[q], ++guard)
                                    consider(q);
                                break;
                            }
                            if (kk == -1) break;
                            slot = (slot + 1) & (HASH_SIZE - 1);
                        }
                    }
        } else {
            for (int q = 0; q < N; ++q) consider(q);
        }
        if (n > NBR_CAP) { atomicOr(s_err, ST_CAPACITY); n = NBR_CAP; }
        sm.nn[pl] = (uint8_t)n;
        // solid sites within the wall-list radius
        int m = wall_list(S, xw, yw, zw, sm.wal + pl * WALL_CAP);
        if (m > WALL_CAP) { atomicOr(s_err, ST_CAPACITY); m = WALL_CAP; }
        sm.nw[pl] = (uint8_t)m;
    }
    __syncthreads();
    if (halo) build_halo<T>(sm, N, p, pl, own, rank, Nc, nhalo);
}

// ---------------------------------------------------------------------------
// The starting Verlet lists of a step for every bead of every chain, one
// warp per bead over the whole GPU.  A block serves up to 8 consecutive beads
// of one chain and first copies that chain's positions into shared memory;
// each warp's 32 lanes then test 32 beads of the chain at a time in ascending
// order and a ballot compacts the hits, so each list comes out sorted, as the
// block builds make it; lane 0 adds the solid sites within the wall-list
// radius.  It reads the positions the step starts from and runs beside the
// gather, so the particle kernel only copies its beads' lists.  Overflows
// latch the capacity status.  Grid: (ceil(max beads / 8), n_real).
// ---------------------------------------------------------------------------
constexpr int LIST_WARPS = 8;

__global__ void __launch_bounds__(32 * LIST_WARPS) k_lists(const Sim S) {
    extern __shared__ __align__(16) float4 lpos[];  // [N] hi, then [N] lo
    const int r = blockIdx.y;
    const int off = S.bead_off[r], N = S.bead_off[r + 1] - off;
    const int first = blockIdx.x * LIST_WARPS;
    if (first >= N) return;  // block-uniform
    float4 *ph = lpos, *plo = lpos + N;
    for (int q = threadIdx.x; q < N; q += blockDim.x) {
        ph[q] = S.r_hi[off + q];
        plo[q] = S.r_lo[off + q];
    }
    __syncthreads();
    const int p = first + (threadIdx.x >> 5);
    if (p >= N) return;  // warp-uniform, after the block's last barrier
    const int lane = threadIdx.x & 31;
    const size_t g = (size_t)(off + p);
    const float fnx = (float)S.bnx, fny = (float)S.ny, fnz = (float)S.nz;
    const float4 mh = ph[p], ml = plo[p];
    uint16_t *lst = S.nbr_g + g * NBR_CAP;
    int n = 0;
    for (int base = 0; base < N; base += 32) {
        const int q = base + lane;
        const int qq = q < N ? q : p;
        const float4 qh = ph[qq], ql = plo[qq];
        const float dx = ff_diff(mh.x, ml.x, qh.x, ql.x, fnx, S.binx), dy = ff_diff(mh.y, ml.y, qh.y, ql.y, fny, S.iny),
                    dz = ff_diff(mh.z, ml.z, qh.z, ql.z, fnz, S.inz);
        const bool hit = q < N && (q < p - 1 || q > p + 1) && within2(dx, dy, dz, S.rl2);
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (hit) {
            const int pos = n + __popc(bal & ((1u << lane) - 1u));
            if (pos < NBR_CAP) lst[pos] = (uint16_t)q;
        }
        n += __popc(bal);
    }
    if (lane == 0) {
        const int m = wall_list(S, ff_wrap(mh.x, ml.x, fnx, S.binx), ff_wrap(mh.y, ml.y, fny, S.iny),
                                ff_wrap(mh.z, ml.z, fnz, S.inz), S.wal_g + g * WALL_CAP);
        if (n > NBR_CAP || m > WALL_CAP) atomicOr(&S.ctrl->status, ST_CAPACITY);
        S.nn_g[g] = min(n, NBR_CAP);
        S.nw_g[g] = min(m, WALL_CAP);
    }
}

cudaError_t launch_lists(const Sim &S, cudaStream_t st) {
    if (S.total_beads == 0 || S.max_beads == 0) return cudaSuccess;
    const dim3 grid((S.max_beads + LIST_WARPS - 1) / LIST_WARPS, S.n_real);
    k_lists<<<grid, 32 * LIST_WARPS, (size_t)32 * S.max_beads, st>>>(S);
    return cudaGetLastError();
}

// Copy beads of other blocks of the chain from their owners' replicas
// (buffer buf, written there before the last cluster barrier) into this
// block's: the halo, or with all = true every bead this block does not own.
// Called by every thread of the block; ends with a block barrier.
__device__ __forceinline__ void pull_beads(cg::cluster_group &cl, const PSmem &sm, int buf, int N, int Nc, int rank,
                                           int c0, bool all, int nhalo) {
    float4 *ph = sm.ph(buf), *plo = sm.pl(buf);
    const int n = all ? N : nhalo;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const uint32_t e = all ? 0u : sm.halo[k];
        const int q = all ? k : (int)(e & 0xffffu);
        const int c = all ? q / Nc : (int)(e >> 16);
        if (c == rank) continue;
        const float4 a = *cl.map_shared_rank(ph + q, c0 + c);
        const float4 b = *cl.map_shared_rank(plo + q, c0 + c);
        ph[q] = a;
        plo[q] = b;
    }
    __syncthreads();
}

// A list rebuild in the MD cycle: with the pull exchange the whole chain is
// first copied into this block's replica, then the block's lists (and halo)
// are built.  Called out of line or inlined.  Out of line, the rare
// rebuild's code stays out of the MD sub-step loop, which then fits the
// instruction cache better (the 400-bead particle kernel: 183 -> 172 us per
// LB step), at the price of a few registers.  Inlined, the kernel keeps its
// register count, which the bead-lanes shapes of the ensemble, sharing SMs
// with the lattice pass, need.
template <int T>
__device__ __forceinline__ void rebuild_body(const Sim &S, const PSmem &sm, int buf, int N, int p, int pl, bool own,
                                             int rank, int Nc, int c0, bool pull, int *clear_flag, int *s_err,
                                             int *nhalo) {
    if (pull) {
        cg::cluster_group cl = cg::this_cluster();
        pull_beads(cl, sm, buf, N, Nc, rank, c0, true, 0);
    }
    build_lists_body<T>(S, sm, buf, N, p, pl, own, rank, Nc, pull, clear_flag, s_err, nhalo);
}
template <int T>
__device__ __noinline__ void rebuild_call(const Sim &S, int nmax, int buf, int N, int p, int pl, bool own,
                                          int rank, int Nc, int c0, bool pull, int *clear_flag, int *s_err,
                                          int *nhalo) {
    // the shared-memory map is laid out again here rather than passed: a
    // PSmem whose address reached this call would live in local memory
    extern __shared__ __align__(16) char smem_raw[];
    PSmem sm;
    psmem_layout(nmax, Nc, spv_noise_slots(S, Nc), &sm, smem_raw);
    rebuild_body<T>(S, sm, buf, N, p, pl, own, rank, Nc, c0, pull, clear_flag, s_err, nhalo);
}
template <int T, bool OUT_OF_LINE>
__device__ __forceinline__ void rebuild(const Sim &S, const PSmem &sm, int nmax, int buf, int N, int p, int pl, bool own,
                                        int rank, int Nc, int c0, bool pull, int *clear_flag, int *s_err, int *nhalo) {
    if constexpr (OUT_OF_LINE) rebuild_call<T>(S, nmax, buf, N, p, pl, own, rank, Nc, c0, pull, clear_flag, s_err, nhalo);
    else rebuild_body<T>(S, sm, buf, N, p, pl, own, rank, Nc, c0, pull, clear_flag, s_err, nhalo);
}

// SM cycles spent in phase k of realization 0 (only while profiling)
__device__ __forceinline__ void phase_mark(const Sim &S, int k, unsigned long long &t) {
    if (S.phase && blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned long long now = clock64();
        atomicAdd(S.phase + k, now - t);
        t = now;
    }
}

// ---------------------------------------------------------------------------
// FP64 block sum of NV values per thread; result valid in thread 0
// ---------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (*red)[NV]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) red[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < NV; ++k) v[k] = 0.0;
        for (int w = 0; w < nw; ++w)
            for (int k = 0; k < NV; ++k) v[k] += red[w][k];
    }
}

__device__ __forceinline__ void sync_all(cg::cluster_group &cl, int C) {
    if (C > 1) cl.sync();
    else __syncthreads();
}

// ---------------------------------------------------------------------------
// the particle kernel (one cluster of C blocks per realization).  VAR 0 and 1
// are the lean forms of the velocity-Verlet cycle without a trajectory
// record, with the push (0) or pull (1) exchange fixed at compile time; VAR
// 2 has every path (exchange from S.md_pull, the SPV integrator, the
// adjoint's trajectory record).  The MD cycle is bound by the latency of its
// dependent sub-steps, and a smaller loop body runs it faster (about 6% on a
// 1000-bead chain over 16 blocks).
// ---------------------------------------------------------------------------
template <int T, bool BWM, int VAR>
__global__ void __launch_bounds__(512, 1) k_particles(const Sim S, const int C, const int Nmax, const int Nc) {
    extern __shared__ __align__(16) char smem_raw[];
    __shared__ int s_flag[2], s_err, s_nhalo;
    PSmem sm;
    psmem_layout(Nmax, Nc, spv_noise_slots(S, Nc), &sm, smem_raw);
    cg::cluster_group cl = cg::this_cluster();
    // this block's part: chain r (-1: an idle block), its rank among the
    // chain's cc blocks, which start at rank c0 of the cluster
    const int4 bm = S.md_map[blockIdx.x];
    const int r = bm.x, rank = bm.y, cc = bm.z, c0 = bm.w;
    const int off = r >= 0 ? S.bead_off[r] : 0;
    const int N = r >= 0 ? S.bead_off[r + 1] - off : 0;
    const int lt = threadIdx.x % T, pl = threadIdx.x / T;
    const int p = rank * Nc + pl;
    const bool own = pl < Nc && p < N;
    const bool owner = own && lt == 0;  // the lane that publishes the bead
    const bool bw = BWM && threadIdx.x >= blockDim.x - 32 * bonded_warps(Nc);  // the warps of the bonded terms
    const int first = rank * Nc, last = min(first + Nc, N) - 1;  // the block's beads
    const bool pull_mode = VAR == 2 ? S.md_pull != 0 : VAR == 1;
    const bool pull = pull_mode && cc > 1;  // block-uniform
    const long long step = S.ctrl->step;
    const float fnx = (float)S.bnx, fny = (float)S.ny, fnz = (float)S.nz;
    unsigned long long tclk = clock64();
    if (threadIdx.x == 0) { s_flag[0] = 0; s_flag[1] = 0; s_err = 0; }

    // replica of the whole chain (both buffers, so that every entry a force
    // term might read holds a finite position) and the state of this lane's bead
    // (up to four of a thread's beads are loaded before any is stored, so
    // that their global loads are in flight together)
    for (int q0 = threadIdx.x; q0 < N; q0 += 4 * blockDim.x) {
        float4 a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = q0 + u * (int)blockDim.x;
            if (q < N) {
                a[u] = S.r_hi[off + q];
                b[u] = S.r_lo[off + q];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = q0 + u * (int)blockDim.x;
            if (q < N) {
                sm.ph(0)[q] = a[u];
                sm.pl(0)[q] = b[u];
                sm.ph(1)[q] = a[u];
                sm.pl(1)[q] = b[u];
            }
        }
    }
    float4 mh = make_float4(0.f, 0.f, 0.f, 0.f), ml = mh;
    float3 v = make_float3(0.f, 0.f, 0.f), up = v;
    if (own) {
        mh = S.r_hi[off + p];
        ml = S.r_lo[off + p];
        const float4 vv = S.v[off + p];
        v = make_float3(vv.x, vv.y, vv.z);
        const float4 uu = S.up[off + p];
        up = make_float3(uu.x, uu.y, uu.z);
    }
    float4 *const trj = VAR == 2 ? S.traj : nullptr;  // trajectory record for the adjoint (usually null)
    const int TB = S.total_beads;
    if (trj && owner) {
        trj[(size_t)traj_slot_hi(S.M, S.Mb, 0) * TB + off + p] = mh;
        trj[(size_t)traj_slot_lo(S.M, S.Mb, 0) * TB + off + p] = ml;
        trj[(size_t)traj_slot_up(S.M, S.Mb) * TB + off + p] = make_float4(up.x, up.y, up.z, 0.f);
    }
    // every block of the cluster is running and initialised before any
    // block writes into another's shared memory
    sync_all(cl, C);
    phase_mark(S, 0, tclk);
    // the block's beads' starting lists, built by k_lists, then the halo.  A
    // bead's lists are NBR_CAP 16-bit and WALL_CAP 32-bit slots, 16-byte
    // aligned in both places: each lane copies its 16-byte chunks of both
    // whole lists, loaded together with the lengths (one round trip to
    // global memory; the slots past the lengths are never read)
    static_assert(NBR_CAP % 8 == 0 && WALL_CAP % 4 == 0, "lists copy in 16-byte chunks");
    if (own) {
        constexpr int NV = NBR_CAP / 8, WV = WALL_CAP / 4;
        constexpr int NL = (NV + T - 1) / T, WL = (WV + T - 1) / T;
        const size_t g = (size_t)(off + p);
        const uint4 *nsrc = reinterpret_cast<const uint4 *>(S.nbr_g + g * NBR_CAP);
        const uint4 *wsrc = reinterpret_cast<const uint4 *>(S.wal_g + g * WALL_CAP);
        uint4 nch[NL], wch[WL];
#pragma unroll
        for (int u = 0; u < NL; ++u)
            if (lt + u * T < NV) nch[u] = nsrc[lt + u * T];
#pragma unroll
        for (int u = 0; u < WL; ++u)
            if (lt + u * T < WV) wch[u] = wsrc[lt + u * T];
        const int n = S.nn_g[g], m = S.nw_g[g];
        uint4 *ndst = reinterpret_cast<uint4 *>(sm.nbr + pl * NBR_CAP);
        uint4 *wdst = reinterpret_cast<uint4 *>(sm.wal + pl * WALL_CAP);
#pragma unroll
        for (int u = 0; u < NL; ++u)
            if (lt + u * T < NV) ndst[lt + u * T] = nch[u];
#pragma unroll
        for (int u = 0; u < WL; ++u)
            if (lt + u * T < WV) wdst[lt + u * T] = wch[u];
        if (lt == 0) {
            sm.nn[pl] = (uint8_t)n;
            sm.nw[pl] = (uint8_t)m;
        }
    }
    __syncthreads();
    if (pull) build_halo<T>(sm, N, p, pl, own, rank, Nc, &s_nhalo);
    phase_mark(S, 1, tclk);

    // MD cycle
    const float dt = 1.0f / (float)S.M, h = 0.5f * dt;
    const float dtb = dt / (float)S.Mb, hb = 0.5f * dtb;
    const float amp = S.kT > 0.0f ? sqrtf(2.0f * S.gamma * S.kT / dt) : 0.0f;
    float3 J = make_float3(0.f, 0.f, 0.f);
    float4 bh = mh, bl = ml;  // position at the last list build
    int buf = 0, t = 0;
    float3 ff = full_force<T, BWM>(S, sm, buf, own, bw, p, pl, N, Nc, first, last, mh, ml, lt);
    // Stochastic position Verlet (integrator 1): the half kicks carry the
    // field only; each sub-step drifts to its mid-point (h/2 for the first,
    // then h: the second half of one sub-step and the first of the next),
    // evaluates the forces there and updates v with the exact
    // Ornstein-Uhlenbeck step v' = c v + (1 - c) u_p + g1 F + sig z; the
    // fluid's impulse is v' - v - h F; a last half drift closes the cycle.
    const bool spv = VAR == 2 && S.integrator == 1;
    for (int sub = 0; sub < S.M; ++sub) {
        float3 xi = make_float3(0.f, 0.f, 0.f);
        if (own && amp > 0.0f && !spv) xi = amp * gauss3(S.seed, S.real_base + (uint32_t)r, (uint32_t)p, step, (uint32_t)sub);
        if (own) {  // first half kick: field + friction + noise (field only for SPV)
            const bool ch = in_channel(S, ff_wrap(mh.x, ml.x, fnx, S.binx), ff_wrap(mh.y, ml.y, fny, S.iny),
                                       ff_wrap(mh.z, ml.z, fnz, S.inz));
            if (trj && lt == 0)
                trj[(size_t)traj_slot_kick(S.M, S.Mb, 2 * sub) * TB + off + p] = make_float4(v.x, v.y, v.z, ch ? 1.f : 0.f);
            if (spv) {
                v.x += h * (ch ? S.E : 0.0f);
            } else {
                const float3 fl = S.gamma * (up - v) + xi;
                v = v + h * (make_float3(ch ? S.E : 0.0f, 0.f, 0.f) + fl);
                J = J + h * fl;
            }
        }
        // SPV: the noise of this outer step's inner steps for the block's
        // beads, drawn by all threads at once (counter t = sub Mb + b, as
        // each inner step would draw it), off the sub-steps' dependent chain
        if (spv && S.spv_sig > 0.0f) {
            __syncthreads();  // the previous outer step's noise has been used
            for (int k = threadIdx.x; k < Nc * S.Mb; k += blockDim.x) {
                const int bl = k / S.Mb, bb = k - bl * S.Mb, q = rank * Nc + bl;
                if (q < N) {
                    const float3 z = gauss3(S.seed, S.real_base + (uint32_t)r, (uint32_t)q, step, (uint32_t)(sub * S.Mb + bb));
                    sm.znz[k] = make_float4(z.x, z.y, z.z, 0.f);
                }
            }
            __syncthreads();
        }
        for (int b = 0; b < S.Mb; ++b, ++t) {
            const int nb = buf ^ 1;
            if (own) {
                if (!spv) v = v + hb * ff;
                const float dr = (spv && b == 0) ? hb : dtb;
                ff_add(mh.x, ml.x, dr * v.x);
                ff_add(mh.y, ml.y, dr * v.y);
                ff_add(mh.z, ml.z, dr * v.z);
                if (trj && lt == 0) {
                    trj[(size_t)traj_slot_hi(S.M, S.Mb, t + 1) * TB + off + p] = mh;
                    trj[(size_t)traj_slot_lo(S.M, S.Mb, t + 1) * TB + off + p] = ml;
                }
                const float3 dd = ffsub(mh, ml, bh, bl);
                const bool moved = dot3(dd, dd) > S.skin_half2;
                // push: the T lanes of a bead share the writes to the cc
                // replicas of its chain; pull: the new position goes into
                // this block's replica, and the lanes share the writes of a
                // rebuild request
                if (pull) {
                    if (lt == 0) {
                        sm.ph(nb)[p] = mh;
                        sm.pl(nb)[p] = ml;
                    }
                    if (moved)
                        for (int c = c0 + lt; c < c0 + cc; c += T) *cl.map_shared_rank(&s_flag[t & 1], c) = 1;
                } else if (cc > 1) {
                    for (int c = c0 + lt; c < c0 + cc; c += T) {
                        *cl.map_shared_rank(sm.ph(nb) + p, c) = mh;
                        *cl.map_shared_rank(sm.pl(nb) + p, c) = ml;
                        if (moved) *cl.map_shared_rank(&s_flag[t & 1], c) = 1;
                    }
                } else if (lt == 0) {
                    sm.ph(nb)[p] = mh;
                    sm.pl(nb)[p] = ml;
                    if (moved) s_flag[t & 1] = 1;
                }
            }
            sync_all(cl, C);
            buf = nb;
            if (s_flag[t & 1]) {
                const unsigned long long t0 = clock64();
                rebuild<T, BWM>(S, sm, Nmax, buf, N, p, pl, own, rank, Nc, c0, pull, &s_flag[t & 1], &s_err, &s_nhalo);
                bh = mh;
                bl = ml;
                if (S.phase && blockIdx.x == 0 && threadIdx.x == 0) {
                    atomicAdd(S.phase + 4, clock64() - t0);  // cycles in rebuilds
                    atomicAdd(S.phase + 5, 1ull);            // rebuilds
                }
            } else if (pull) {
                pull_beads(cl, sm, buf, N, Nc, rank, c0, false, s_nhalo);
            }
            const float3 F = full_force<T, BWM>(S, sm, buf, own, bw, p, pl, N, Nc, first, last, mh, ml, lt);
            if (own) {
                if (spv) {
                    float3 z = make_float3(0.f, 0.f, 0.f);
                    if (S.spv_sig > 0.0f) {
                        const float4 zz = sm.znz[pl * S.Mb + b];
                        z = make_float3(zz.x, zz.y, zz.z);
                    }
                    const float3 vn = S.spv_c * v + (1.0f - S.spv_c) * up + S.spv_g1 * F + S.spv_sig * z;
                    J = J + (vn - v - dtb * F);
                    v = vn;
                } else {
                    ff = F;
                    v = v + hb * ff;
                }
            }
        }
        if (own) {
            if (spv) {  // the last half drift of the cycle
                ff_add(mh.x, ml.x, hb * v.x);
                ff_add(mh.y, ml.y, hb * v.y);
                ff_add(mh.z, ml.z, hb * v.z);
            }
            // second half kick with the same noise (field only for SPV)
            const bool ch = in_channel(S, ff_wrap(mh.x, ml.x, fnx, S.binx), ff_wrap(mh.y, ml.y, fny, S.iny),
                                       ff_wrap(mh.z, ml.z, fnz, S.inz));
            if (trj && lt == 0)
                trj[(size_t)traj_slot_kick(S.M, S.Mb, 2 * sub + 1) * TB + off + p] = make_float4(v.x, v.y, v.z, ch ? 1.f : 0.f);
            if (spv) {
                v.x += h * (ch ? S.E : 0.0f);
            } else {
                const float3 fl = S.gamma * (up - v) + xi;
                v = v + h * (make_float3(ch ? S.E : 0.0f, 0.f, 0.f) + fl);
                J = J + h * fl;
            }
        }
    }
    // pull: no block leaves while another may still be reading its replica
    // (push: the last writes into another block's shared memory came before
    // the last sub-step's cluster barrier)
    if (pull_mode) sync_all(cl, C);
    if (owner) sm.jbuf[pl] = make_float4(J.x, J.y, J.z, 0.f);
    __syncthreads();
    phase_mark(S, 2, tclk);

    // spread -W J onto the fluid corners of the starting position, with the
    // (site, weight) pairs the gather kernel recorded: one thread per pair
    {
        const size_t ns = (size_t)S.ns;
        const int nown = max(0, min(Nc, N - rank * Nc));
        for (int k = threadIdx.x; k < 8 * nown; k += blockDim.x) {
            const size_t pair = (size_t)(off + rank * Nc) * 8 + k;
            const int gnode = S.pair_node[pair];
            if (gnode < 0) continue;
            const float W = S.pair_w[pair];
            const float4 Jq = sm.jbuf[k >> 3];
            const size_t base = (size_t)r * 2 * ns + (size_t)gnode;  // = (r*3 + 0)*ns + site
            atomicAdd(S.G + base, (unsigned long long)__float2ll_rn(-W * Jq.x * FIX_SCALE_F));
            atomicAdd(S.G + base + ns, (unsigned long long)__float2ll_rn(-W * Jq.y * FIX_SCALE_F));
            atomicAdd(S.G + base + 2 * ns, (unsigned long long)__float2ll_rn(-W * Jq.z * FIX_SCALE_F));
        }
    }
    if (owner) {
        ff_norm(mh.x, ml.x);
        ff_norm(mh.y, ml.y);
        ff_norm(mh.z, ml.z);
        S.r_hi[off + p] = mh;
        S.r_lo[off + p] = ml;
        S.v[off + p] = make_float4(v.x, v.y, v.z, 0.f);
        S.J[off + p] = make_float4(J.x, J.y, J.z, 0.f);
        if (trj) trj[(size_t)traj_slot_J(S.M, S.Mb) * TB + off + p] = make_float4(J.x, J.y, J.z, 0.f);
        if (!isfinite(mh.x + mh.y + mh.z + v.x + v.y + v.z)) atomicOr(&s_err, ST_NONFINITE);
    }
    // this barrier collects the error flags
    __syncthreads();
    phase_mark(S, 3, tclk);
    if (threadIdx.x == 0 && s_err) atomicOr(&S.ctrl->status, s_err);
}

// Launch (n_fit null) or, with n_fit, report how many clusters of the shape
// can be resident at once (0: the device cannot schedule one).
template <int T>
static cudaError_t launch_particles_t(const Sim &S, const MdShape &m, cudaStream_t st, int *n_fit) {
    // the lean kernels where no SPV cycle and no trajectory record is asked for
    const bool full = S.integrator == 1 || S.traj != nullptr;
    auto kern = full ? (m.bw ? k_particles<T, true, 2> : k_particles<T, false, 2>)
                : S.md_pull ? (m.bw ? k_particles<T, true, 1> : k_particles<T, false, 1>)
                            : (m.bw ? k_particles<T, true, 0> : k_particles<T, false, 0>);
    size_t dyn = m.launch_smem;
    if (dyn > m.smem) {  // reserving: the opt-in maximum counts static and dynamic shared memory together
        cudaFuncAttributes fa;
        cudaError_t ea = cudaFuncGetAttributes(&fa, kern);
        if (ea != cudaSuccess) return ea;
        dyn = dyn > fa.sharedSizeBytes ? max(m.smem, dyn - fa.sharedSizeBytes) : m.smem;
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    if (m.C > 8) {  // clusters above the portable size of 8 are opt-in
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(S.md_clusters * m.C);
    cfg.blockDim = dim3(m.threads);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = m.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (n_fit) return cudaOccupancyMaxActiveClusters(n_fit, (void *)kern, &cfg);
    return cudaLaunchKernelEx(&cfg, kern, S, m.C, max(S.max_beads, 1), m.Nc);
}

static cudaError_t particles_dispatch(const Sim &S, cudaStream_t st, int *n_fit) {
    const MdShape m = md_shape(S);
    switch (m.T) {
        case 1: return launch_particles_t<1>(S, m, st, n_fit);
        case 2: return launch_particles_t<2>(S, m, st, n_fit);
        case 8: return launch_particles_t<8>(S, m, st, n_fit);
        default: return launch_particles_t<4>(S, m, st, n_fit);
    }
}

cudaError_t launch_particles(const Sim &S, const void *, cudaStream_t st) {
    if (S.total_beads == 0 || S.md_clusters == 0) return cudaSuccess;
    return particles_dispatch(S, st, nullptr);
}

cudaError_t particles_clusters_fit(const Sim &S, int *n_fit) {
    *n_fit = 0;
    if (S.total_beads == 0 || S.md_clusters == 0) return cudaSuccess;
    return particles_dispatch(S, 0, n_fit);
}

// ---------------------------------------------------------------------------
// bead observables at the current state (one block per realization)
// ---------------------------------------------------------------------------
template <int PREC>
__global__ void __launch_bounds__(1024) k_bead_observables(const Sim S, const void *__restrict__ Av) {
    using T = typename PopT<PREC>::T;
    extern __shared__ __align__(16) char smem_raw[];
    __shared__ double red[32][9];
    float4 *ph = reinterpret_cast<float4 *>(smem_raw);
    float4 *plo = ph + blockDim.x;
    float4 *ups = plo + blockDim.x;
    const int r = blockIdx.x;
    const int off = S.bead_off[r];
    const int N = S.bead_off[r + 1] - off;
    const int p = threadIdx.x;
    const bool own = p < N;
    const T *A = reinterpret_cast<const T *>(Av) + (size_t)r * Q * S.ps;
    const float fnx = (float)S.bnx, fny = (float)S.ny, fnz = (float)S.nz;
    float4 mh = make_float4(0.f, 0.f, 0.f, 0.f), ml = mh, vv = mh;
    if (own) {
        mh = S.r_hi[off + p];
        ml = S.r_lo[off + p];
        vv = S.v[off + p];
        ph[p] = mh;
        plo[p] = ml;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int q = warp; q < N; q += nwarps) {
        const float4 qh = ph[q], ql = plo[q];
        int node, xi, xc0;
        float W;
        const float3 u = gather_warp(S, A, ff_wrap(qh.x, ql.x, fnx, S.binx), ff_wrap(qh.y, ql.y, fny, S.iny),
                                     ff_wrap(qh.z, ql.z, fnz, S.inz), node, W, xi, xc0);
        if ((threadIdx.x & 31) == 0) ups[q] = make_float4(u.x, u.y, u.z, 0.f);
    }
    __syncthreads();
    const double X = (double)mh.x + (double)ml.x, Y = (double)mh.y + (double)ml.y, Z = (double)mh.z + (double)ml.z;
    const bool tr = own && S.wall_x >= 0 && X > (double)S.wall_x + 0.5;
    double a[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (own) {
        const float4 u = ups[p];
        const bool ch = in_channel(S, ff_wrap(mh.x, ml.x, fnx, S.binx), ff_wrap(mh.y, ml.y, fny, S.iny),
                                   ff_wrap(mh.z, ml.z, fnz, S.inz));
        a[0] = vv.x; a[1] = vv.y; a[2] = vv.z;
        a[3] = X; a[4] = Y; a[5] = Z;
        a[6] = tr ? 1.0 : 0.0;
        a[7] = (double)S.gamma * ((double)vv.x * u.x + (double)vv.y * u.y + (double)vv.z * u.z);
        a[8] = ch ? (double)S.E * vv.x : 0.0;
    }
    block_sum<9>(a, red);
    __shared__ double s_sum[9];
    if (threadIdx.x == 0)
        for (int k = 0; k < 9; ++k) s_sum[k] = a[k];
    // centres of the translocated / untranslocated parts
    double c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (own) {
        const int o = tr ? 4 : 0;
        c[o] = X; c[o + 1] = Y; c[o + 2] = Z; c[o + 3] = 1.0;
    }
    __shared__ double red8[32][8];
    block_sum<8>(c, red8);
    __shared__ double s_c[8];
    if (threadIdx.x == 0)
        for (int k = 0; k < 8; ++k) s_c[k] = c[k];
    __syncthreads();
    double g2[2] = {0, 0};
    if (own) {
        const int o = tr ? 4 : 0;
        const double n = s_c[o + 3];
        const double dx = X - s_c[o] / n, dy = Y - s_c[o + 1] / n, dz = Z - s_c[o + 2] / n;
        g2[tr ? 1 : 0] = dx * dx + dy * dy + dz * dz;
    }
    __shared__ double red2[32][2];
    block_sum<2>(g2, red2);
    if (threadIdx.x == 0) {
        lbmd_obs *o = S.obs + r;
        // fluid sums of the observables pass of the lattice kernel (run before this)
        long long *acc = S.fsum + 4 * ((size_t)S.n_real + r);
        const double unit = fix_unit(FIXD_FLUID);
        o->mass = S.n_fluid + (double)acc[0] * unit;
        o->p_fluid[0] = (double)acc[1] * unit;
        o->p_fluid[1] = (double)acc[2] * unit;
        o->p_fluid[2] = (double)acc[3] * unit;
        acc[0] = 0; acc[1] = 0; acc[2] = 0; acc[3] = 0;
        o->p_beads[0] = s_sum[0]; o->p_beads[1] = s_sum[1]; o->p_beads[2] = s_sum[2];
        const double inv = N > 0 ? 1.0 / N : 0.0;
        o->com[0] = s_sum[3] * inv; o->com[1] = s_sum[4] * inv; o->com[2] = s_sum[5] * inv;
        o->n_translocated = s_sum[6];
        o->dWH_dt = s_sum[7];
        o->dWE_dt = s_sum[8];
        o->rg_untranslocated = s_c[3] > 0 ? sqrt(g2[0] / s_c[3]) : 0.0;
        o->rg_translocated = s_c[7] > 0 ? sqrt(g2[1] / s_c[7]) : 0.0;
    }
}

cudaError_t launch_bead_observables(const Sim &S, const void *A, cudaStream_t st) {
    const int threads = max(32, ((S.max_beads + 31) / 32) * 32);
    const size_t smem = 48 * (size_t)threads;
    if (S.precision == LBMD_FP16DEV) k_bead_observables<1><<<S.n_real, threads, smem, st>>>(S, A);
    else k_bead_observables<0><<<S.n_real, threads, smem, st>>>(S, A);
    return cudaGetLastError();
}

}  // namespace lbmd
