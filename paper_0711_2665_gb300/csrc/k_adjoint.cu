// k_adjoint.cu -- reverse-mode (adjoint) kernels of the coupled LB-MD step.
//
// The forward step n maps (A^n, r^n, v^n) to (A^{n+1}, r^{n+1}, v^{n+1}),
// with A the stored post-collision deviations (f* - w) and f^n = pull(A^n):
//   gather   u_p = sum_k W_k(r^n) u(f^n(x_k))            (trilinear, Sec. II)
//   MD       M half-kick / M^b velocity-Verlet / half-kick cycles (Eq. 22)
//            with the friction gamma (u_p - v) and noise (Eqs. 12, 13, 15),
//            accumulating the impulse J_p
//   spread   G(x_k) = -sum_p W_k(r^p) J_p                 (Eq. 8)
//   lattice  A^{n+1}(x) = f - omega (f - f_eq(f)) + 3 w_i c_i . (G + g)
//                                                          (Eqs. 4, 5, 9)
// Given the adjoints of the outputs (lam_A^{n+1}, lam_r, lam_v) the three
// kernels below return those of the inputs:
//   k_sc_adjoint:    lam_A^n = pull^T [ (d f*/d f)^T lam_A^{n+1} ] at every
//                    fluid site; the transposed pull writes each lam_f_i(x)
//                    to the one (population, site) the pull read f_i(x) from;
//   k_bead_adjoint:  lam_G at the corners -> lam_J; the MD cycle in reverse
//                    (force Jacobian-vector products with dual numbers);
//                    lam_u_p -> lam_r through the weights, and lam_u at the
//                    corner sites (2^40 fixed-point atomics); FP64 sums of
//                    dL/dgamma and dL/dE;
//   k_adj_fixup:     lam_f_i(x) += lam_u(x) . (c_i - u(x)) / rho(x) at the
//                    corner sites, through the same transposed pull.
// The bead kernel reads the trajectory the forward particle kernel recorded
// while the step was replayed from a checkpoint.
#include "lbmd_internal.cuh"

namespace lbmd {

// ---------------------------------------------------------------------------
// dual numbers: value and tangent (directional derivative)
// ---------------------------------------------------------------------------
struct Du {
    float v, d;
};
__device__ __forceinline__ Du du(float v, float d = 0.f) { return Du{v, d}; }
__device__ __forceinline__ Du operator+(Du a, Du b) { return Du{a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Du operator-(Du a, Du b) { return Du{a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Du operator*(Du a, Du b) { return Du{a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Du operator*(float s, Du a) { return Du{s * a.v, s * a.d}; }
// The tangents feed a first-order sensitivity; fast reciprocals and square
// roots (relative error ~1e-7) are ample for it.
__device__ __forceinline__ Du operator/(Du a, Du b) {
    const float ib = __frcp_rn(b.v);
    const float q = a.v * ib;
    return Du{q, (a.d - q * b.d) * ib};
}
__device__ __forceinline__ Du dsqrt(Du a) {
    const float r = rsqrtf(a.v);
    const float s = a.v * r;
    return Du{s, 0.5f * a.d * r};
}
__device__ __forceinline__ Du drsqrt(Du a) {
    const float r = rsqrtf(a.v);
    return Du{r, -0.5f * a.d * r * r * r};
}
// atan2(y, x) for y >= 0 (the angle of the angular term): value from the
// forward kernel's polynomial, d = (x dy - y dx) / (x^2 + y^2)
__device__ __forceinline__ Du datan2(Du y, Du x) {
    return Du{atan_pos(y.v, x.v), (x.v * y.d - y.v * x.d) * __frcp_rn(x.v * x.v + y.v * y.v)};
}

struct Du3 {
    Du x, y, z;
};
__device__ __forceinline__ Du3 du3(float3 v, float3 t) { return Du3{du(v.x, t.x), du(v.y, t.y), du(v.z, t.z)}; }
__device__ __forceinline__ Du3 operator+(Du3 a, Du3 b) { return Du3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ Du3 operator-(Du3 a, Du3 b) { return Du3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ Du3 operator*(Du s, Du3 a) { return Du3{s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ Du ddot(Du3 a, Du3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ Du3 dcross(Du3 a, Du3 b) {
    return Du3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ float3 tangent(Du3 a) { return make_float3(a.x.d, a.y.d, a.z.d); }

__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 add3(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 mul3(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3f(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
// unwrapped difference of two float-float positions (bonded neighbours)
__device__ __forceinline__ float3 ffsub3(float4 ah, float4 al, float4 bh, float4 bl) {
    return make_float3((ah.x - bh.x) + (al.x - bl.x), (ah.y - bh.y) + (al.y - bl.y), (ah.z - bh.z) + (al.z - bl.z));
}

// ---------------------------------------------------------------------------
// tangent of the conservative forces on bead p along the displacement field w
// (positions hi/lo and w of every bead of the chain in shared memory):
// sum_q dF_p/dr_q w_q.  Terms as in the forward kernel: harmonic bonds
// (Eq. 19), the angular term kappa phi^2 / 2 at the angles p-1, p, p+1, WCA
// between beads (|p - q| >= 2, minimum image) and with solid sites (Eq. 14).
// ---------------------------------------------------------------------------
// angle between u and w: D1 = A dcos/du, D2 = A dcos/dw, A = kappa phi / sin phi
__device__ __forceinline__ void bend_dual(Du3 b1, Du3 b2, float kappa, Du3 &D1, Du3 &D2) {
    const Du l1s = ddot(b1, b1), l2s = ddot(b2, b2), dt = ddot(b1, b2);
    const Du3 cr = dcross(b1, b2);
    const Du cr2 = ddot(cr, cr);
    const Du inv12 = drsqrt(l1s * l2s);
    const Du c = dt * inv12;
    Du A = du(c.v > 0.0f ? kappa : 0.0f);
    if (cr2.v > 0.0f) {
        const Du crn = dsqrt(cr2);
        const Du sn = crn * inv12;
        if (sn.v > 1e-6f) {
            const Du phi = datan2(crn, dt);
            A = (kappa * phi) / sn;
        }
    }
    D1 = A * ((inv12 * b2) - ((c / l1s) * b1));
    D2 = A * ((inv12 * b1) - ((c / l2s) * b2));
}

// tangent of coef(r2) d for the WCA force coef(r2) d, coef = 24 eps (2 s^12/r^14 - s^6/r^8)
__device__ __forceinline__ float3 wca_tangent(float3 d, float3 dd, float eps, float sig2) {
    const float r2 = dot3f(d, d);
    const float ir2 = __frcp_rn(r2), sr2 = sig2 * ir2;
    const float sr6 = sr2 * sr2 * sr2;
    const float coef = 24.0f * eps * (2.0f * sr6 * sr6 - sr6) * ir2;
    const float dcoef = 24.0f * eps * (-14.0f * sr6 * sr6 + 4.0f * sr6) * ir2 * ir2 * (2.0f * dot3f(d, dd));
    return add3(mul3(dcoef, d), mul3(coef, dd));
}

// Pair list of one lane of bead p for one outer MD step: the beads q with
// q % T == lt within the list radius (ADJ_LANE_CAP entries; a count of
// ADJ_ALL_PAIRS means the list overflowed and every bead of the lane's
// residue class is a candidate).
constexpr int ADJ_LANE_CAP = 16;
constexpr int ADJ_ALL_PAIRS = 0xffff;
// Wall list of one lane: packed solid-site coordinates x | y << 12 | z << 22
// (ADJ_WALL_CAP entries; ADJ_ALL_PAIRS: take the lane's share of the 4x4x4
// box mask at every evaluation).
constexpr int ADJ_WALL_CAP = 8;

// Lane lt's part of the tangent of the conservative force on bead p along the
// displacement field w (positions hi/lo and w of the chain in shared memory):
// sum over its terms of dF_p/dr_q w_q.  Terms as in the forward kernel: the
// bonded triples (a, b, c) = (p+s-2, p+s-1, p+s) for s = lt, lt+T, .. < 3 with
// the angle at b and, for s < 2, the bond b-c (Eq. 19); WCA with the lane's
// listed beads (|p - q| >= 2, minimum image) and with every T-th solid site of
// the 4x4x4 box around the bead's cell (Eq. 14).
template <int T>
__device__ __forceinline__ float3 force_tangent_part(const Sim &S, const float4 *__restrict__ sh, const float4 *__restrict__ sl,
                                                     const float4 *__restrict__ sw, int p, int N, int lt,
                                                     const uint16_t *__restrict__ lst, int nl,
                                                     const uint32_t *__restrict__ wlst, int nwl) {
    const float4 mh = sh[p], ml = sl[p];
    const float3 wp = f3(sw[p]);
    float3 Tn = make_float3(0.f, 0.f, 0.f);
    for (int s = lt; s < 3; s += T) {
        const int ia = p + s - 2, ib = p + s - 1, ic = p + s;
        const bool bond_ok = s < 2 && ib >= 0 && ic < N;
        const bool ang_ok = ia >= 0 && ic < N && S.kappa != 0.0f;
        if (!bond_ok && !ang_ok) continue;
        const int ja = ia >= 0 ? ia : ib;  // ia < 0 only when the angle is unused
        const Du3 u = du3(ffsub3(sh[ib], sl[ib], sh[ja], sl[ja]), sub3(f3(sw[ib]), f3(sw[ja])));  // r_b - r_a
        const Du3 w = du3(ffsub3(sh[ic], sl[ic], sh[ib], sl[ib]), sub3(f3(sw[ic]), f3(sw[ib])));  // r_c - r_b
        if (bond_ok) {  // p = c (s = 0): -k(|w| - r0) w/|w|;  p = b (s = 1): +...
            const Du len = dsqrt(ddot(w, w));
            const Du coef = du(S.k_bond) - (S.k_bond * S.r0) * (du(1.f) / len);
            const float3 t = tangent(coef * w);
            Tn = s == 0 ? sub3(Tn, t) : add3(Tn, t);
        }
        if (ang_ok) {  // share of the angle at b on p = c, b, a: +D2, D1 - D2, -D1
            Du3 D1, D2;
            bend_dual(u, w, S.kappa, D1, D2);
            if (s == 0) Tn = add3(Tn, tangent(D2));
            else if (s == 1) Tn = add3(Tn, tangent(D1 - D2));
            else Tn = sub3(Tn, tangent(D1));
        }
    }
    const float fnx = (float)S.nx, fny = (float)S.ny, fnz = (float)S.nz;
    const bool all = nl == ADJ_ALL_PAIRS;
    const int nq = all ? (N - lt + T - 1) / T : nl;
    for (int k = 0; k < nq; ++k) {
        const int q = all ? lt + k * T : (int)lst[k];
        if (q >= p - 1 && q <= p + 1) continue;
        const float4 qh = sh[q], ql = sl[q];
        const float3 d = make_float3(ff_diff(mh.x, ml.x, qh.x, ql.x, fnx, S.inx), ff_diff(mh.y, ml.y, qh.y, ql.y, fny, S.iny),
                                     ff_diff(mh.z, ml.z, qh.z, ql.z, fnz, S.inz));
        if (dot3f(d, d) < S.lj_rc2) Tn = add3(Tn, wca_tangent(d, sub3(wp, f3(sw[q])), S.lj_eps, S.lj_sig2));
    }
    if (nwl != ADJ_ALL_PAIRS) {  // the lane's listed solid sites
        for (int k = 0; k < nwl; ++k) {
            const uint32_t pk = wlst[k];
            const float3 d = make_float3(ff_diff(mh.x, ml.x, (float)(pk & 0xfffu), 0.f, fnx, S.inx),
                                         ff_diff(mh.y, ml.y, (float)((pk >> 12) & 0x3ffu), 0.f, fny, S.iny),
                                         ff_diff(mh.z, ml.z, (float)(pk >> 22), 0.f, fnz, S.inz));
            if (dot3f(d, d) < S.wall_rc2) Tn = add3(Tn, wca_tangent(d, wp, S.wall_eps, S.wall_sig2));
        }
        return Tn;
    }
    // solid sites of the 4x4x4 box around the bead's cell (it holds every
    // site within the cut-off, which is below 2); lane lt takes every T-th
    const float xw = ff_wrap(mh.x, ml.x, fnx, S.inx), yw = ff_wrap(mh.y, ml.y, fny, S.iny), zw = ff_wrap(mh.z, ml.z, fnz, S.inz);
    const int cx0 = (int)floorf(xw), cy0 = (int)floorf(yw), cz0 = (int)floorf(zw);
    unsigned long long mm = __ldg(S.wallmask + cx0 + S.nx * (cy0 + S.ny * cz0));
    for (int j = 0; mm; ++j) {
        const int bit = __ffsll((long long)mm) - 1;
        mm &= mm - 1;
        if (j % T != lt) continue;
        const int X = wrap_any(cx0 + (bit & 3) - 1, S.nx), Y = wrap_any(cy0 + ((bit >> 2) & 3) - 1, S.ny),
                  Z = wrap_any(cz0 + (bit >> 4) - 1, S.nz);
        const float3 d = make_float3(ff_diff(mh.x, ml.x, (float)X, 0.f, fnx, S.inx), ff_diff(mh.y, ml.y, (float)Y, 0.f, fny, S.iny),
                                     ff_diff(mh.z, ml.z, (float)Z, 0.f, fnz, S.inz));
        if (dot3f(d, d) < S.wall_rc2) Tn = add3(Tn, wca_tangent(d, wp, S.wall_eps, S.wall_sig2));
    }
    return Tn;
}

// sum over the T consecutive lanes of a bead (fixed butterfly: every lane
// gets the same, deterministic sum)
template <int T>
__device__ __forceinline__ float3 lane_sum(float3 v) {
#pragma unroll
    for (int o = 1; o < T; o <<= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
        v.z += __shfl_xor_sync(0xffffffffu, v.z, o);
    }
    return v;
}

// ---------------------------------------------------------------------------
// renormalised trilinear weights at a bead and their gradient in r:
//   W_k = m_k w_k / sum_j m_j w_j,  w_k = prod_a (f_a or 1 - f_a),
//   dW_k/dr_a = (m_k dw_k/dr_a - W_k sum_j m_j dw_j/dr_a) / sum_j m_j w_j
// ---------------------------------------------------------------------------
struct Corners {
    int node[8];
    float W[8];
    float3 dW[8];
};

__device__ __forceinline__ void corners_with_gradient(const Sim &S, float xw, float yw, float zw, Corners &c) {
    const int x0 = (int)floorf(xw), y0 = (int)floorf(yw), z0 = (int)floorf(zw);
    const float f[3] = {xw - (float)x0, yw - (float)y0, zw - (float)z0};
    float raw[8], sum = 0.f;
    float3 dsum = make_float3(0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int a = k & 1, b = (k >> 1) & 1, d = k >> 2;
        const int xi = wrapi(x0 + a, S.nx), yi = wrapi(y0 + b, S.ny), zi = wrapi(z0 + d, S.nz);
        c.node[k] = xi + S.nx * (yi + S.ny * zi);
        const float m = (__ldg(S.link + c.node[k]) & SOLID_BIT) ? 0.0f : 1.0f;
        const float fx = a ? f[0] : 1.0f - f[0], fy = b ? f[1] : 1.0f - f[1], fz = d ? f[2] : 1.0f - f[2];
        const float sx = a ? 1.0f : -1.0f, sy = b ? 1.0f : -1.0f, sz = d ? 1.0f : -1.0f;
        raw[k] = m * fx * fy * fz;
        c.dW[k] = make_float3(m * sx * fy * fz, m * fx * sy * fz, m * fx * fy * sz);
        if (S.interp == 1) {  // nearest grid point: piecewise constant, gradient 0
            raw[k] = m * ((a == (f[0] >= 0.5f) && b == (f[1] >= 0.5f) && d == (f[2] >= 0.5f)) ? 1.0f : 0.0f);
            c.dW[k] = make_float3(0.f, 0.f, 0.f);
        }
        sum += raw[k];
        dsum = add3(dsum, c.dW[k]);
    }
    const float inv = sum > 0.0f ? 1.0f / sum : 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        c.W[k] = raw[k] * inv;
        c.dW[k] = mul3(inv, sub3(c.dW[k], mul3(c.W[k], dsum)));
    }
}

// rho and u at site s of realization base A (FP32 deviations), from the
// populations the pull delivers there (bounce-back where the link word says)
__device__ __forceinline__ void pulled_moments(const Sim &S, const float *__restrict__ A, int s, float &rho, float3 &u) {
    const int x = s % S.nx, y = (s / S.nx) % S.ny, z = s / (S.nx * S.ny);
    const uint32_t lm = __ldg(S.link + s);
    float m = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const uint32_t src = (uint32_t)(wrapi(x - cx(i), S.nx) + S.nx * (wrapi(y - cy(i), S.ny) + S.ny * wrapi(z - cz(i), S.nz)));
        const uint32_t idx = ((lm >> i) & 1u) ? (uint32_t)opp(i) * S.ps + (uint32_t)s : (uint32_t)i * S.ps + src;
        const float h = __ldcg(A + idx);
        m += h;
        jx += (float)cx(i) * h;
        jy += (float)cy(i) * h;
        jz += (float)cz(i) * h;
    }
    rho = 1.0f + m;
    u = rho > 0.0f ? make_float3(jx / rho, jy / rho, jz / rho) : make_float3(0.f, 0.f, 0.f);
}

// ---------------------------------------------------------------------------
// lattice adjoint: lam_A^n = pull^T [ (1 - omega) lam* + omega J_eq^T lam* ]
// with lam* = lam_A^{n+1}(x) and J_eq = d f_eq / d f through rho and u:
//   (J_eq^T lam)_k = a + c_k . (3 b + 9 d - 3 s0 u),
//   s0 = sum_i w_i lam_i,  b = sum_i w_i lam_i c_i,  d = sum_i w_i lam_i (c_i.u) c_i,
//   a  = sum_i w_i lam_i (1 - 9/2 (c_i.u)^2 + 3/2 u.u).
// The transposed pull stores lam_f_k(x) where the pull read f_k(x) from:
// A_k(x - c_k), or A_opp(k)(x) when that link bounces back.  The map is a
// bijection on the fluid (population, site) pairs, so no two sites write the
// same word.  Block (32, by) over x, y; each thread walks zc planes.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_sc_adjoint(const Sim S, const float *__restrict__ Av, const float *__restrict__ Lin,
                                                    float *__restrict__ Lout, const int zc, const int nzb) {
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int r = blockIdx.z / nzb;
    const int z0 = (blockIdx.z - r * nzb) * zc;
    const int nx = S.nx, ny = S.ny, nz = S.nz;
    if (x >= nx || y >= ny) return;
    const uint32_t ps = (uint32_t)S.ps;
    const size_t base = (size_t)r * Q * ps;
    const float *__restrict__ A = Av + base;
    const float *__restrict__ Li = Lin + base;
    float *__restrict__ Lo = Lout + base;
    const float om = S.omega;
    const int xv0 = (x == 0 ? nx - 1 : x - 1), xv2 = (x == nx - 1 ? 0 : x + 1);
    const int yv0 = (y == 0 ? ny - 1 : y - 1), yv2 = (y == ny - 1 ? 0 : y + 1);
    const int zend = min(z0 + zc, nz);
    for (int z = z0; z < zend; ++z) {
        const int zv0 = (z == 0 ? nz - 1 : z - 1), zv2 = (z == nz - 1 ? 0 : z + 1);
        const int s = x + nx * (y + ny * z);
        const uint32_t lm = S.tileflag[blockIdx.x + S.nxt * (y + ny * z)] ? __ldg(S.link + s) : 0u;
        if (lm & SOLID_BIT) continue;
        uint32_t idx[Q];
        float m = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int sx = cx(i) == 1 ? xv0 : (cx(i) == -1 ? xv2 : x);
            const int sy = cy(i) == 1 ? yv0 : (cy(i) == -1 ? yv2 : y);
            const int sz = cz(i) == 1 ? zv0 : (cz(i) == -1 ? zv2 : z);
            const uint32_t src = (uint32_t)(sx + nx * (sy + ny * sz));
            idx[i] = ((lm >> i) & 1u) ? (uint32_t)opp(i) * ps + (uint32_t)s : (uint32_t)i * ps + src;
            const float h = __ldg(A + idx[i]);
            m += h;
            jx += (float)cx(i) * h;
            jy += (float)cy(i) * h;
            jz += (float)cz(i) * h;
        }
        const float rho = 1.0f + m, ir = 1.0f / rho;
        const float ux = jx * ir, uy = jy * ir, uz = jz * ir;
        const float uu = ux * ux + uy * uy + uz * uz;
        float lam[Q];
        float s0 = 0.f, a = 0.f, bx = 0.f, by = 0.f, bz = 0.f, dx = 0.f, dy = 0.f, dz = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            lam[i] = __ldg(Li + (uint32_t)i * ps + (uint32_t)s);
            const float wl = wq(i) * lam[i];
            const float cu = (float)cx(i) * ux + (float)cy(i) * uy + (float)cz(i) * uz;
            s0 += wl;
            a += wl * (1.0f - 4.5f * cu * cu + 1.5f * uu);
            bx += (float)cx(i) * wl; by += (float)cy(i) * wl; bz += (float)cz(i) * wl;
            const float wlc = wl * cu;
            dx += (float)cx(i) * wlc; dy += (float)cy(i) * wlc; dz += (float)cz(i) * wlc;
        }
        const float qx = 3.0f * bx + 9.0f * dx - 3.0f * s0 * ux;
        const float qy = 3.0f * by + 9.0f * dy - 3.0f * s0 * uy;
        const float qz = 3.0f * bz + 9.0f * dz - 3.0f * s0 * uz;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const float jt = a + (float)cx(k) * qx + (float)cy(k) * qy + (float)cz(k) * qz;
            Lo[idx[k]] = (1.0f - om) * lam[k] + om * jt;
        }
    }
}

cudaError_t launch_sc_adjoint(const Sim &S, const void *A, const float *Lin, float *Lout, int by, int zc, cudaStream_t st) {
    const int nzb = (S.nz + zc - 1) / zc;
    dim3 grid((S.nx + 31) / 32, (S.ny + by - 1) / by, nzb * S.n_real);
    k_sc_adjoint<<<grid, dim3(32, by), 0, st>>>(S, reinterpret_cast<const float *>(A), Lin, Lout, zc, nzb);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// bead adjoint: one block per realization, one thread per bead.
// ---------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_sum_d(double (&v)[NV], double (*red)[NV]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
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

// One block per chain; T lanes per bead split the corner terms, the bonded
// triples, the pair list and the wall sites, and hold the bead's adjoint
// state identically (lane_sum gives every lane the same sums).
template <int T, int MAXT>
__global__ void __launch_bounds__(MAXT) k_bead_adjoint(const Sim S, const float *__restrict__ Av, const float *__restrict__ Lin,
                                                       const float4 *__restrict__ trj, float4 *__restrict__ lam_r,
                                                       float4 *__restrict__ lam_v, unsigned long long *__restrict__ LU,
                                                       int *__restrict__ adj_node, double *__restrict__ dpar,
                                                       const long long step, const int Nmax) {
    extern __shared__ __align__(16) float4 smq[];
    __shared__ double red[32][2];
    float4 *sh = smq, *sl = smq + Nmax, *sw = smq + 2 * Nmax;
    float *sd = reinterpret_cast<float *>(smq + 3 * Nmax);                 // [Nmax] displacement bound
    uint32_t *wal = reinterpret_cast<uint32_t *>(sd + ((Nmax + 3) & ~3));  // [Nmax][T][ADJ_WALL_CAP]
    uint16_t *nbr = reinterpret_cast<uint16_t *>(wal + (size_t)Nmax * T * ADJ_WALL_CAP);  // [Nmax][T][ADJ_LANE_CAP]
    const int r = blockIdx.x;
    const int off = S.bead_off[r];
    const int N = S.bead_off[r + 1] - off;
    const int lt = threadIdx.x % T;
    const int p = threadIdx.x / T;
    const bool own = p < N;
    const bool lead = own && lt == 0;  // the lane that writes the bead's results
    const int g = off + (own ? p : 0);
    const int TB = S.total_beads, M = S.M, Mb = S.Mb;
    const size_t ns = (size_t)S.ns;
    const float *A = Av + (size_t)r * Q * S.ps;
    const float *L = Lin + (size_t)r * Q * S.ps;
    const float fnx = (float)S.nx, fny = (float)S.ny, fnz = (float)S.nz;

    float3 lr = make_float3(0.f, 0.f, 0.f), lv = lr, up = lr;
    if (own) {
        lr = f3(lam_r[g]);
        lv = f3(lam_v[g]);
        up = f3(trj[(size_t)traj_slot_up(M, Mb) * TB + g]);
    }
    // corner sites, weights and weight gradients at the step's start position
    // (recomputed where needed rather than held through the MD loop)
    auto corners = [&](Corners &cn) {
        const float4 h0 = trj[(size_t)traj_slot_hi(M, Mb, 0) * TB + g];
        const float4 l0 = trj[(size_t)traj_slot_lo(M, Mb, 0) * TB + g];
        corners_with_gradient(S, ff_wrap(h0.x, l0.x, fnx, S.inx), ff_wrap(h0.y, l0.y, fny, S.iny),
                              ff_wrap(h0.z, l0.z, fnz, S.inz), cn);
    };

    // spread: G(x_k) -= W_k J  =>  lam_J -= W_k lam_G(x_k), lam_r -= dW_k (J . lam_G(x_k)),
    // with lam_G(x) = sum_i 3 w_i c_i lam_A_i(x) (source of Eq. 9); lane lt
    // takes the corners k = lt, lt + T, ...
    float3 lJ = make_float3(0.f, 0.f, 0.f), lrw = lJ;
    if (own) {
        Corners cn;
        corners(cn);
        const float3 J = f3(trj[(size_t)traj_slot_J(M, Mb) * TB + g]);
#pragma unroll 1
        for (int k = lt; k < 8; k += T) {
            if (cn.W[k] == 0.0f && cn.dW[k].x == 0.0f && cn.dW[k].y == 0.0f && cn.dW[k].z == 0.0f) continue;
            float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const float l3 = 3.0f * wq(i) * __ldcg(L + (uint32_t)i * S.ps + (uint32_t)cn.node[k]);
                gx += (float)cx(i) * l3;
                gy += (float)cy(i) * l3;
                gz += (float)cz(i) * l3;
            }
            const float3 lg = make_float3(gx, gy, gz);
            lJ = sub3(lJ, mul3(cn.W[k], lg));
            lrw = sub3(lrw, mul3(dot3f(J, lg), cn.dW[k]));
        }
    }
    lJ = lane_sum<T>(lJ);
    lrw = lane_sum<T>(lrw);

    // the MD cycle in reverse
    const float dt = 1.0f / (float)M, h = 0.5f * dt;
    const float dtb = dt / (float)Mb, hb = 0.5f * dtb;
    const float gam = S.gamma;
    const bool noisy = S.kT > 0.0f && gam > 0.0f;
    const float amp = noisy ? sqrtf(2.0f * gam * S.kT / dt) : 0.0f;
    float3 lup = make_float3(0.f, 0.f, 0.f);
    double dg = 0.0, de = 0.0;
    auto load_positions = [&](int t) {
        for (int q = threadIdx.x; q < N; q += blockDim.x) {
            sh[q] = trj[(size_t)traj_slot_hi(M, Mb, t) * TB + off + q];
            sl[q] = trj[(size_t)traj_slot_lo(M, Mb, t) * TB + off + q];
        }
    };
    // reverse of v' = v + h (E chi x^ + gamma (u_p - v) + xi), J' = J + h (gamma (u_p - v) + xi)
    auto kick = [&](int k, float3 xi) {
        const float4 kv = trj[(size_t)traj_slot_kick(M, Mb, k) * TB + g];
        const float3 vb = f3(kv);
        const float3 s = add3(lv, lJ);
        const float3 dxi = noisy ? mul3(0.5f / gam, xi) : make_float3(0.f, 0.f, 0.f);
        dg += (double)h * (double)dot3f(add3(sub3(up, vb), dxi), s);
        de += (double)h * (double)kv.w * (double)lv.x;
        lup = add3(lup, mul3(h * gam, s));
        lv = sub3(mul3(1.0f - h * gam, lv), mul3(h * gam, lJ));
    };
    // Pair lists for the sub-steps of one outer step, from the recorded
    // positions: a pair closer than the cut-off at any of its sub-steps is
    // closer than rc + D_p + D_q at its start, D the bead's largest
    // displacement during the outer step.
    int nl = 0, nwl = 0;
    uint16_t *my = nbr + ((size_t)(own ? p : 0) * T + lt) * ADJ_LANE_CAP;
    uint32_t *myw = wal + ((size_t)(own ? p : 0) * T + lt) * ADJ_WALL_CAP;
    const float rc = sqrtf(S.lj_rc2);
    auto build_list = [&](int sub) {
        float dm = 0.0f;
        const int t0 = sub * Mb;
        if (own) {
            const float4 ah = trj[(size_t)traj_slot_hi(M, Mb, t0) * TB + g], al = trj[(size_t)traj_slot_lo(M, Mb, t0) * TB + g];
            for (int t = t0 + 1 + lt; t <= t0 + Mb; t += T) {
                const float3 d = ffsub3(trj[(size_t)traj_slot_hi(M, Mb, t) * TB + g], trj[(size_t)traj_slot_lo(M, Mb, t) * TB + g], ah, al);
                dm = fmaxf(dm, dot3f(d, d));
            }
        }
#pragma unroll
        for (int o = 1; o < T; o <<= 1) dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, o));  // over the bead's lanes
        if (own && lt == 0) sd[p] = sqrtf(dm) * 1.0001f + 1e-6f;
        load_positions(t0);
        __syncthreads();
        nl = 0;
        if (own) {
            const float4 mh = sh[p], ml = sl[p];
            const float dp = sd[p];
            for (int q = lt; q < N; q += T) {
                if (q >= p - 1 && q <= p + 1) continue;
                const float4 qh = sh[q], ql = sl[q];
                const float3 d = make_float3(ff_diff(mh.x, ml.x, qh.x, ql.x, fnx, S.inx), ff_diff(mh.y, ml.y, qh.y, ql.y, fny, S.iny),
                                             ff_diff(mh.z, ml.z, qh.z, ql.z, fnz, S.inz));
                const float rl = rc + dp + sd[q];
                if (dot3f(d, d) < rl * rl) {
                    if (nl < ADJ_LANE_CAP) my[nl] = (uint16_t)q;
                    ++nl;
                }
            }
            if (nl > ADJ_LANE_CAP) nl = ADJ_ALL_PAIRS;
            // solid sites closer than rc_w + D_p at the start: the 4x4x4 box of
            // the start cell holds every site within rc_w of the later
            // positions while D_p < 0.85 (rc_w < 1.15); else the mask is
            // walked at every evaluation
            nwl = 0;
            if (dp < 0.85f && S.wall_rc2 < 1.3225f) {
                const float xw = ff_wrap(mh.x, ml.x, fnx, S.inx), yw = ff_wrap(mh.y, ml.y, fny, S.iny),
                            zw = ff_wrap(mh.z, ml.z, fnz, S.inz);
                const int cx0 = (int)floorf(xw), cy0 = (int)floorf(yw), cz0 = (int)floorf(zw);
                unsigned long long mm = __ldg(S.wallmask + cx0 + S.nx * (cy0 + S.ny * cz0));
                const float rw = sqrtf(S.wall_rc2) + dp;
                for (int j = 0; mm; ++j) {
                    const int bit = __ffsll((long long)mm) - 1;
                    mm &= mm - 1;
                    if (j % T != lt) continue;
                    const int X = wrap_any(cx0 + (bit & 3) - 1, S.nx), Y = wrap_any(cy0 + ((bit >> 2) & 3) - 1, S.ny),
                              Z = wrap_any(cz0 + (bit >> 4) - 1, S.nz);
                    const float3 d = make_float3(ff_diff(mh.x, ml.x, (float)X, 0.f, fnx, S.inx),
                                                 ff_diff(mh.y, ml.y, (float)Y, 0.f, fny, S.iny),
                                                 ff_diff(mh.z, ml.z, (float)Z, 0.f, fnz, S.inz));
                    if (dot3f(d, d) < rw * rw) {
                        if (nwl < ADJ_WALL_CAP) myw[nwl] = (uint32_t)X | ((uint32_t)Y << 12) | ((uint32_t)Z << 22);
                        ++nwl;
                    }
                }
                if (nwl > ADJ_WALL_CAP) nwl = ADJ_ALL_PAIRS;
            } else {
                nwl = ADJ_ALL_PAIRS;
            }
        }
        __syncthreads();
    };
    auto tangent_all = [&]() {
        const float3 part = own ? force_tangent_part<T>(S, sh, sl, sw, p, N, lt, my, nl, myw, nwl) : make_float3(0.f, 0.f, 0.f);
        return lane_sum<T>(part);
    };
    for (int sub = M - 1; sub >= 0; --sub) {
        build_list(sub);
        load_positions((sub + 1) * Mb);
        float3 xi = make_float3(0.f, 0.f, 0.f);
        if (own && noisy) xi = mul3(amp, gauss3(S.seed, S.real_base + (uint32_t)r, (uint32_t)p, step, (uint32_t)sub));
        if (own) kick(2 * sub + 1, xi);
        for (int b = Mb - 1; b >= 0; --b) {
            const int t = sub * Mb + b;
            // the positions r_t of the second evaluation, fetched now so that
            // their latency passes during the first (one bead per thread:
            // the block has at least N threads)
            const int q = threadIdx.x;
            float4 ph = make_float4(0.f, 0.f, 0.f, 0.f), pl = ph;
            if (q < N) {
                ph = trj[(size_t)traj_slot_hi(M, Mb, t) * TB + off + q];
                pl = trj[(size_t)traj_slot_lo(M, Mb, t) * TB + off + q];
            }
            // v' = v_h + hb F(r_{t+1})
            if (lead) sw[p] = make_float4(lv.x, lv.y, lv.z, 0.f);
            __syncthreads();
            float3 jw = tangent_all();
            __syncthreads();
            lr = add3(lr, mul3(hb, jw));
            // r_{t+1} = r_t + dtb v_h
            lv = add3(lv, mul3(dtb, lr));
            // v_h = v + hb F(r_t)
            if (q < N) {
                sh[q] = ph;
                sl[q] = pl;
            }
            if (lead) sw[p] = make_float4(lv.x, lv.y, lv.z, 0.f);
            __syncthreads();
            jw = tangent_all();
            __syncthreads();
            lr = add3(lr, mul3(hb, jw));
        }
        if (own) kick(2 * sub, xi);
    }

    // gather: u_p = sum_k W_k u(x_k)  =>  lam_r += dW_k (u(x_k) . lam_up); lam_u(x_k) += W_k lam_up
    float3 lrg = make_float3(0.f, 0.f, 0.f);
    if (own) {
        Corners cn;
        corners(cn);
#pragma unroll 1
        for (int k = lt; k < 8; k += T) {
            int gnode = -1;
            if (cn.W[k] > 0.0f || cn.dW[k].x != 0.0f || cn.dW[k].y != 0.0f || cn.dW[k].z != 0.0f) {
                float rho;
                float3 u;
                pulled_moments(S, A, cn.node[k], rho, u);
                lrg = add3(lrg, mul3(dot3f(u, lup), cn.dW[k]));
                if (cn.W[k] > 0.0f) {
                    const size_t b0 = (size_t)r * 3 * ns + (size_t)cn.node[k];
                    atomicAdd(LU + b0, (unsigned long long)__float2ll_rn(cn.W[k] * lup.x * FIX_SCALE_F));
                    atomicAdd(LU + b0 + ns, (unsigned long long)__float2ll_rn(cn.W[k] * lup.y * FIX_SCALE_F));
                    atomicAdd(LU + b0 + 2 * ns, (unsigned long long)__float2ll_rn(cn.W[k] * lup.z * FIX_SCALE_F));
                    gnode = (int)((size_t)r * ns + (size_t)cn.node[k]);
                }
            }
            adj_node[(size_t)g * 8 + k] = gnode;
        }
    }
    lrg = lane_sum<T>(lrg);
    if (lead) {
        lr = add3(add3(lr, lrg), lrw);
        lam_r[g] = make_float4(lr.x, lr.y, lr.z, 0.f);
        lam_v[g] = make_float4(lv.x, lv.y, lv.z, 0.f);
    }
    double acc[2] = {lead ? dg : 0.0, lead ? de : 0.0};
    block_sum_d<2>(acc, red);
    if (threadIdx.x == 0) {
        dpar[2 * r] += acc[0];
        dpar[2 * r + 1] += acc[1];
    }
}

// lanes per bead: 4 up to 128 beads, 2 up to 256, 1 above (at most 512
// threads per block, 128 registers; chains above 512 beads take 1024)
static int adj_lanes(int nmax) { return nmax <= 128 ? 4 : (nmax <= 256 ? 2 : 1); }

size_t bead_adjoint_smem(const Sim &S) {
    const size_t n = (size_t)max(S.max_beads, 1);
    const size_t T = (size_t)adj_lanes(S.max_beads);
    return 3 * 16 * n + 4 * ((n + 3) & ~(size_t)3) + 4 * ADJ_WALL_CAP * T * n + ((2 * ADJ_LANE_CAP * T * n + 15) & ~(size_t)15);
}

template <int T, int MAXT>
static cudaError_t launch_bead_adjoint_t(const Sim &S, const float *A, const float *Lin, const float4 *trj, float4 *lam_r,
                                         float4 *lam_v, unsigned long long *LU, int *adj_node, double *dpar, long long step,
                                         cudaStream_t st) {
    const int threads = max(32, ((S.max_beads * T + 31) / 32) * 32);
    const size_t smem = bead_adjoint_smem(S);
    cudaError_t e = cudaFuncSetAttribute(k_bead_adjoint<T, MAXT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_bead_adjoint<T, MAXT><<<S.n_real, threads, smem, st>>>(S, A, Lin, trj, lam_r, lam_v, LU, adj_node, dpar, step,
                                                             max(S.max_beads, 1));
    return cudaGetLastError();
}

cudaError_t launch_bead_adjoint(const Sim &S, const void *A, const float *Lin, const float4 *trj, float4 *lam_r, float4 *lam_v,
                                unsigned long long *LU, int *adj_node, double *dpar, long long step, cudaStream_t st) {
    const float *Af = reinterpret_cast<const float *>(A);
    switch (adj_lanes(S.max_beads)) {
    case 4: return launch_bead_adjoint_t<4, 512>(S, Af, Lin, trj, lam_r, lam_v, LU, adj_node, dpar, step, st);
    case 2: return launch_bead_adjoint_t<2, 512>(S, Af, Lin, trj, lam_r, lam_v, LU, adj_node, dpar, step, st);
    default:
        if (S.max_beads <= 512) return launch_bead_adjoint_t<1, 512>(S, Af, Lin, trj, lam_r, lam_v, LU, adj_node, dpar, step, st);
        return launch_bead_adjoint_t<1, 1024>(S, Af, Lin, trj, lam_r, lam_v, LU, adj_node, dpar, step, st);
    }
}

// ---------------------------------------------------------------------------
// corner-site fix-up: lam_f_i(x) += lam_u(x) . (c_i - u(x)) / rho(x)  (u = j / rho),
// added through the transposed pull.  The first (bead, corner) pair to stamp a
// site with this step's (negative) tag serves it; distinct sites have
// distinct targets, so the read-modify-writes do not race.  The stamps are
// the adjoint's own (the forward replay beside it stamps S.stamp).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_adj_fixup(const Sim S, const float *__restrict__ Av, float *__restrict__ Lout,
                                                   const int *__restrict__ adj_node, unsigned long long *__restrict__ LU,
                                                   int *__restrict__ stamp, const int tag) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 8 * S.total_beads) return;
    const int gnode = adj_node[k];
    if (gnode < 0 || atomicExch(stamp + gnode, tag) == tag) return;
    const size_t ns = (size_t)S.ns;
    const int r = (int)(gnode / ns);
    const int s = (int)(gnode - (size_t)r * ns);
    unsigned long long *Ur = LU + (size_t)r * 3 * ns + s;
    const float3 lu = make_float3((float)(long long)Ur[0] * FIX_INV_SCALE_F, (float)(long long)Ur[ns] * FIX_INV_SCALE_F,
                                  (float)(long long)Ur[2 * ns] * FIX_INV_SCALE_F);
    Ur[0] = 0ull; Ur[ns] = 0ull; Ur[2 * ns] = 0ull;
    const float *A = Av + (size_t)r * Q * S.ps;
    float *Lo = Lout + (size_t)r * Q * S.ps;
    float rho;
    float3 u;
    pulled_moments(S, A, s, rho, u);
    if (!(rho > 0.0f)) return;
    const float ir = 1.0f / rho;
    const float lu_u = dot3f(lu, u);
    const int x = s % S.nx, y = (s / S.nx) % S.ny, z = s / (S.nx * S.ny);
    const uint32_t lm = __ldg(S.link + s);
    uint32_t idx[Q];
    float old[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {  // all loads before any store (one L2 round trip)
        const uint32_t src = (uint32_t)(wrapi(x - cx(i), S.nx) + S.nx * (wrapi(y - cy(i), S.ny) + S.ny * wrapi(z - cz(i), S.nz)));
        idx[i] = ((lm >> i) & 1u) ? (uint32_t)opp(i) * S.ps + (uint32_t)s : (uint32_t)i * S.ps + src;
        old[i] = __ldcg(Lo + idx[i]);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float dl = ((float)cx(i) * lu.x + (float)cy(i) * lu.y + (float)cz(i) * lu.z - lu_u) * ir;
        Lo[idx[i]] = old[i] + dl;
    }
}

cudaError_t launch_adj_fixup(const Sim &S, const void *A, float *Lout, const int *adj_node, unsigned long long *LU, int *stamp,
                             int tag,
                             cudaStream_t st) {
    if (S.total_beads == 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (8 * S.total_beads + threads - 1) / threads;
    k_adj_fixup<<<blocks, threads, 0, st>>>(S, reinterpret_cast<const float *>(A), Lout, adj_node, LU, stamp, tag);
    return cudaGetLastError();
}

}  // namespace lbmd
