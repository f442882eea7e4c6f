// lbmd_api.cu -- host side of the C ABI declared in include/lbmd.h: argument
// checks, the layout of the caller's device buffer, geometry preprocessing,
// the per-step launch sequence (particle kernel and stream-collide kernel
// concurrently on two streams, then the source pass), CUDA-graph replay,
// per-kernel event timing and the tile autotuner.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lbmd_internal.cuh"

using namespace lbmd;

namespace {

constexpr int K_GATHER = 0, K_PARTICLES = 1, K_STREAM_COLLIDE = 2, K_SOURCE = 3, K_SC_ADJOINT = 4,
              K_BEAD_ADJOINT = 5, K_ADJ_FIXUP = 6, K_BEAD_DIAG = 7, K_LISTS = 8, K_COUNT = 9;
const char *KNAMES[] = {"gather", "particles", "stream_collide", "source", "sc_adjoint", "bead_adjoint",
                               "adj_fixup", "bead_diag", "lists"};
static_assert(sizeof(KNAMES) / sizeof(KNAMES[0]) == K_COUNT, "one name per kernel");
constexpr double SKIN = 0.6;  // Verlet-list skin (lattice units); 0.4 and 0.8 measured slower

struct Layout {
    size_t blink, bwallmask, xsend_lo, xsend_hi, xrecv_lo, xrecv_hi;  // slab mode only (else 0)
    size_t popA, popB, staging, link, wallmask, tileflag, solid, G, stamp;
    size_t r_hi, r_lo, v, up, J, pair_node, pair_w, bead_real, bead_off, bsnap, fsum, ring, obs, tl, ctrl, loopc, snap, md_map, phase, total;
    size_t nbr_g, wal_g, nn_g, nw_g;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct ProfRec {
    int kernel;
    cudaEvent_t a, b;
};

}  // namespace

struct lbmd_handle {
    lbmd_config cfg;
    Sim S;
    char *dbuf = nullptr;
    size_t dbytes = 0;
    Layout L;
    void *popA = nullptr, *popB = nullptr;
    float *staging = nullptr;
    std::vector<int32_t> offsets;
    int total_beads = 0;
    cudaStream_t st = nullptr, aux = nullptr, aux2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join2 = nullptr, ev_pre = nullptr, ev_lists = nullptr;
    cudaEvent_t ev_lists_cap = nullptr;  // ev_lists inside a stream capture (a captured record cannot be waited on outside it)
    // the adjoint's backward sweep: its streams (the bead adjoint on baux),
    // fork/join, start, and per record buffer the ends of replay and backward
    cudaStream_t bst = nullptr, baux = nullptr;
    cudaEvent_t ev_bfork = nullptr, ev_bjoin = nullptr, ev_bstart = nullptr, ev_rep[2] = {nullptr, nullptr},
                ev_bwd[2] = {nullptr, nullptr};
    int by = 8, zc = 8;   // by = 0: the tensor-copy lattice kernel with zc row groups per block
    CUtensorMap tmap[2];  // the two population buffers (at L.popA, L.popB) as 5-D tensors
    bool tma_ok = false;  // tmap encoded and the lattice fits the tensor-copy kernel
    bool overlap = true;  // particle kernel concurrent with the lattice pass
    bool md_fixed = false;  // particle-kernel shape set by the caller (the autotuner leaves it)
    int md_exchange = 0;    // chain exchange: 0 the autotuner's choice, 1 push, 2 pull
    int md_bonded = 0;      // bonded terms: 0 the autotuner's choice, 1 every bead's lanes, 2 bonded warps
    int md_reserve = 0;     // SMs of the particle kernel: 0 the autotuner's choice, 1 shared, 2 reserved
    int graph_steps = 0;
    cudaGraphExec_t gexec = nullptr;
    void *graph_A = nullptr;  // population buffer that was "A" when the graph was captured
    cudaGraphExec_t lexec = nullptr;  // device-side loop of two-step bodies (lbmd_step_loop)
    void *loop_A = nullptr;
    bool capturing = false;
    bool profiling = false;
    // The starting Verlet lists of the next step: lists_ready means a k_lists
    // launch for the current bead positions is queued on the particle stream
    // (ev_lists marks its end).  Every write of bead positions outside a step
    // clears it.  lists_in_capture: that launch belongs to the stream capture
    // under way.
    bool lists_ready = false;
    bool lists_in_capture = false;
    std::vector<ProfRec> pending;
    std::vector<cudaEvent_t> free_events;
    double prof_ms[K_COUNT] = {};
    long long prof_n[K_COUNT] = {};
    long long launches = 0;
    long long host_step = 0;
    std::string err;
};

namespace {

lbmd_status fail(lbmd_handle *h, lbmd_status s, const std::string &msg) {
    if (h) h->err = msg;
    return s;
}

lbmd_status cuda_fail(lbmd_handle *h, cudaError_t e, const char *where) {
    cudaGetLastError();  // a failed call leaves no error for a later launch check to pick up
    return fail(h, LBMD_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                      \
    do {                                                              \
        cudaError_t e__ = (call);                                     \
        if (e__ != cudaSuccess) return cuda_fail(h, e__, #call);      \
    } while (0)

bool config_ok(const lbmd_config *c, const int32_t *off, std::string &why) {
    if (!c) { why = "null config"; return false; }
    if (c->nx < 1 || c->ny < 1 || c->nz < 1) { why = "lattice dimensions must be >= 1"; return false; }
    if (c->nx > 4096 || c->ny > 1024 || c->nz > 1024) { why = "lattice limited to 4096 x 1024 x 1024"; return false; }
    const double ns = (double)c->nx * c->ny * c->nz;
    if ((ns + 128.0) * LBMD_Q >= 2147483647.0) { why = "19 * sites must stay below 2^31 per realization"; return false; }
    if (c->n_real < 1 || (double)c->n_real * ns >= 2147483647.0) { why = "n_real must be >= 1 and n_real * sites < 2^31"; return false; }
    if (!(c->tau > 0.5)) { why = "tau must be > 1/2"; return false; }
    if (c->md_outer < 1 || c->md_inner < 1) { why = "md_outer and md_inner must be >= 1"; return false; }
    if (c->precision != LBMD_FP32 && c->precision != LBMD_FP16DEV) { why = "unknown precision"; return false; }
    if (c->real_base < 0 || (double)c->real_base + c->n_real > 4294967295.0) { why = "real_base out of range"; return false; }
    if (c->interp != 0 && c->interp != 1) { why = "interp must be 0 (trilinear) or 1 (nearest grid point)"; return false; }
    if (c->integrator != 0 && c->integrator != 1) { why = "integrator must be 0 (velocity Verlet) or 1 (SPV)"; return false; }
    if (!(c->lb_kT >= 0.0) || !std::isfinite(c->lb_kT)) { why = "lb_kT must be finite and >= 0"; return false; }
    if (c->wall_x < -1 || c->wall_x >= c->nx) { why = "wall_x must be -1 or inside [0, nx)"; return false; }
    if (c->pore_h < 0 || c->pore_h > c->ny || c->pore_h > c->nz) { why = "pore_h out of range"; return false; }
    if (!(c->lj_sigma > 0) || !(c->wall_sigma > 0) || c->lj_eps < 0 || c->wall_eps < 0) { why = "WCA sigma must be > 0, eps >= 0"; return false; }
    if (c->gamma < 0 || c->kT < 0 || c->k_bond < 0) { why = "gamma, kT, k_bond must be >= 0"; return false; }
    if (c->slab_nx < 0 || c->slab_nx > c->nx) { why = "slab_nx must be in [0, nx]"; return false; }
    if (c->slab_nx > 0) {
        if (c->slab_nx < 2) { why = "a slab holds at least 2 planes"; return false; }
        if (c->slab_x0 < 0 || c->slab_x0 >= c->nx) { why = "slab_x0 must be inside [0, nx)"; return false; }
        if (c->n_real != 1) { why = "slab mode takes one realization"; return false; }
        if (c->lb_kT != 0.0) { why = "slab mode runs without the fluctuating fluid"; return false; }
    }
    if (!off) { why = "null bead_offsets"; return false; }
    if (off[0] != 0) { why = "bead_offsets[0] must be 0"; return false; }
    if (off[c->n_real] > 0 && (c->nx < 4 || c->ny < 4 || c->nz < 4)) {
        why = "a lattice holding beads needs at least 4 sites per axis";
        return false;
    }
    for (int r = 0; r < c->n_real; ++r) {
        const int n = off[r + 1] - off[r];
        if (n < 0) { why = "bead_offsets must be non-decreasing"; return false; }
        if (n > LBMD_MAX_BEADS_PER_REALIZATION) { why = "more than 1024 beads in a realization"; return false; }
    }
    return true;
}

// Stride between the 19 population arrays of a lattice: the site count
// rounded up to 64, so that every array starts on a 128-byte boundary in
// both precisions.
size_t pop_stride(size_t ns) { return (ns + 63) / 64 * 64; }

// x planes of the handle's populations: the lattice, or a slab with its
// ghost planes (one on the left, two on the right)
int local_nx(const lbmd_config *c) { return c->slab_nx > 0 ? c->slab_nx + 3 : c->nx; }

Layout layout_of(const lbmd_config *c, int total_beads) {
    Layout L;
    const int nxl = local_nx(c);
    const size_t ns = (size_t)nxl * c->ny * c->nz;
    const size_t esz = c->precision == LBMD_FP16DEV ? 2 : 4;
    const size_t npop = (size_t)c->n_real * LBMD_Q * pop_stride(ns);
    const size_t nxt = (nxl + 31) / 32;
    const size_t nb = (size_t)std::max(total_beads, 1);
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
    L.popA = take(npop * esz);
    L.popB = take(npop * esz);
    L.staging = take((size_t)c->n_real * LBMD_Q * ns * 4);
    L.link = take(ns * 4);
    L.wallmask = take(ns * 8);
    L.tileflag = take(nxt * c->ny * c->nz);
    L.solid = take(ns);
    L.G = take((size_t)c->n_real * 3 * ns * 8);
    L.stamp = take((size_t)c->n_real * ns * 4);
    L.r_hi = take(nb * 16);
    L.r_lo = take(nb * 16);
    L.v = take(nb * 16);
    L.up = take(nb * 16);
    L.J = take(nb * 16);
    L.pair_node = take(nb * 8 * 4);
    L.pair_w = take(nb * 8 * 4);
    L.bead_real = take(nb * 4);
    L.bead_off = take((size_t)(c->n_real + 1) * 4);
    L.bsnap = take(nb * 48);
    L.fsum = take((size_t)c->n_real * 8 * sizeof(long long));
    L.ring = take((size_t)c->n_real * LBMD_DIAG_RING * sizeof(lbmd_diag));
    L.obs = take((size_t)c->n_real * sizeof(lbmd_obs));
    L.tl = take((size_t)c->n_real * sizeof(lbmd_transloc));
    L.ctrl = take(sizeof(Ctrl));
    L.loopc = take(sizeof(unsigned int));
    L.snap = take(nb * 48);  // bead state saved while the autotuner times particle shapes
    // chain placement of the particle kernel: the current shape's and a trial
    // shape's (autotuner); at most one cluster of MAX_CLUSTER blocks per chain
    L.md_map = take(2 * (size_t)c->n_real * MAX_CLUSTER * sizeof(int4));
    L.phase = take(PHASES * sizeof(unsigned long long));
    L.nbr_g = take(nb * NBR_CAP * 2);
    L.wal_g = take(nb * WALL_CAP * 4);
    L.nn_g = take(nb * 4);
    L.nw_g = take(nb * 4);
    L.blink = L.bwallmask = L.xsend_lo = L.xsend_hi = L.xrecv_lo = L.xrecv_hi = 0;
    if (c->slab_nx > 0) {  // the whole lattice's geometry for the beads; the exchanged planes
        const size_t gns = (size_t)c->nx * c->ny * c->nz;
        const size_t plane = (size_t)LBMD_Q * c->ny * c->nz * esz;
        L.blink = take(gns * 4);
        L.bwallmask = take(gns * 8);
        L.xsend_lo = take(2 * plane);
        L.xsend_hi = take(plane);
        L.xrecv_lo = take(plane);
        L.xrecv_hi = take(2 * plane);
    }
    L.total = o;
    return L;
}

cudaEvent_t get_event(lbmd_handle *h) {
    if (!h->free_events.empty()) {
        cudaEvent_t e = h->free_events.back();
        h->free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

lbmd_status resolve_profile(lbmd_handle *h) {
    if (h->pending.empty()) return LBMD_OK;
    CK(cudaStreamSynchronize(h->st));
    CK(cudaStreamSynchronize(h->aux));
    CK(cudaStreamSynchronize(h->aux2));
    for (auto &p : h->pending) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, p.a, p.b));
        h->prof_ms[p.kernel] += ms;
        h->prof_n[p.kernel] += 1;
        h->free_events.push_back(p.a);
        h->free_events.push_back(p.b);
    }
    h->pending.clear();
    return LBMD_OK;
}

struct ProfScope {
    lbmd_handle *h;
    int k;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(lbmd_handle *h_, int k_, cudaStream_t s_) : h(h_), k(k_), s(s_) {
        if (h->profiling && !h->capturing) {
            a = get_event(h);
            b = get_event(h);
            cudaEventRecord(a, s);
        }
    }
    ~ProfScope() {
        if (a) {
            cudaEventRecord(b, s);
            h->pending.push_back({k, a, b});
        }
    }
};

// Placement of the chains in the particle kernel's clusters of C blocks of
// Nc beads: chain r takes ceil(N_r / Nc) consecutive blocks of one cluster,
// first fit over the chains in decreasing length (ties by index), so that
// short chains share a cluster instead of each holding C blocks.  A chain's
// arithmetic does not depend on how many blocks share it.  Realizations
// without beads get no block; blocks left over in a cluster idle.  Returns
// the number of clusters; map gets C entries per cluster.
int pack_chains(const std::vector<int32_t> &off, int C, int Nc, std::vector<int4> &map) {
    const int R = (int)off.size() - 1;
    std::vector<int> order;
    for (int r = 0; r < R; ++r)
        if (off[r + 1] > off[r]) order.push_back(r);
    auto blocks = [&](int r) { return std::max(1, (off[r + 1] - off[r] + Nc - 1) / Nc); };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return blocks(a) > blocks(b); });
    std::vector<int> fill;                      // blocks used per cluster
    std::vector<int4> place;                    // (r, cluster, first block, blocks)
    for (int r : order) {
        const int c = std::min(blocks(r), C);
        size_t k = 0;
        while (k < fill.size() && fill[k] + c > C) ++k;
        if (k == fill.size()) fill.push_back(0);
        place.push_back(make_int4(r, (int)k, fill[k], c));
        fill[k] += c;
    }
    map.assign(fill.size() * (size_t)C, make_int4(-1, 0, 1, 0));
    for (size_t k = 0; k < fill.size(); ++k)
        for (int j = 0; j < C; ++j) map[k * C + j].w = j;  // idle blocks: a chain of their own
    for (const int4 &pl : place)
        for (int j = 0; j < pl.w; ++j) map[(size_t)pl.y * C + pl.z + j] = make_int4(pl.x, j, pl.w, pl.z);
    return (int)fill.size();
}

// Upload the placement for shape m into map region `region` (0: current, 1:
// trial) and point S at it.  Ordered on the main stream, after every step
// already enqueued (their particle kernels have joined it).
lbmd_status upload_md_map(lbmd_handle *h, Sim &S, int region) {
    const MdShape m = md_shape(S);
    std::vector<int4> map;
    const int nc = pack_chains(h->offsets, m.C, m.Nc, map);
    int4 *dst = (int4 *)(h->dbuf + h->L.md_map) + (size_t)region * h->cfg.n_real * MAX_CLUSTER;
    if (!map.empty()) CK(cudaMemcpyAsync(dst, map.data(), map.size() * sizeof(int4), cudaMemcpyHostToDevice, h->st));
    S.md_map = dst;
    S.md_clusters = nc;
    return LBMD_OK;
}

// One coupled step: the gather runs alone (its latency-bound loads would queue
// behind the lattice pass's traffic), then the particle kernel (aux stream)
// and the bead diagnostics (aux2) run concurrently with the stream-collide
// kernel (main), then the source, which also completes the diagnostics row.
// The lattice pass A -> B with tile shape (by, zc): by = 0 is the kernel fed
// by tensor copies, with the map of whichever buffer is A now.
cudaError_t lattice_pass(lbmd_handle *h, const Sim &S, int by, int zc, bool diag) {
    if (by == 0) {
        const CUtensorMap &m = h->popA == (void *)(h->dbuf + h->L.popA) ? h->tmap[0] : h->tmap[1];
        return launch_stream_collide_tma(S, m, h->popA, h->popB, zc, diag, h->st);
    }
    if (by < 0) return launch_stream_collide_x2(S, h->popA, h->popB, -by, zc, diag, h->st);
    return launch_stream_collide(S, h->popA, h->popB, by, zc, diag, h->st);
}

// The two population buffers as 5-D tensors (x, y, z, link, realization) of
// the storage type, one-row boxes, for the tensor-copy lattice kernel.  The
// encoder comes from the driver through the runtime (no driver library is
// linked).  Leaves tma_ok false where the lattice does not fit the kernel or
// the driver lacks the call.
void encode_tensor_maps(lbmd_handle *h) {
    h->tma_ok = false;
    if (!tma_lattice_ok(h->S)) return;
    typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                    const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return;
    }
    const bool f16 = h->cfg.precision == LBMD_FP16DEV;
    const cuuint64_t esz = f16 ? 2 : 4;
    const Sim &S = h->S;
    const cuuint64_t dims[5] = {(cuuint64_t)S.nx, (cuuint64_t)S.ny, (cuuint64_t)S.nz, (cuuint64_t)LBMD_Q,
                                (cuuint64_t)S.n_real};
    const cuuint64_t strides[4] = {(cuuint64_t)S.nx * esz, (cuuint64_t)S.nx * S.ny * esz, (cuuint64_t)S.ps * esz,
                                   (cuuint64_t)LBMD_Q * S.ps * esz};
    const cuuint32_t box[5] = {(cuuint32_t)S.nx, 1, 1, 1, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    void *bufs[2] = {h->dbuf + h->L.popA, h->dbuf + h->L.popB};
    for (int k = 0; k < 2; ++k) {
        const CUresult r = ((EncodeTiled)fn)(&h->tmap[k], f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                                             5, bufs[k], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return;
    }
    if (prepare_stream_collide_tma(S) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    h->tma_ok = true;
}

// Kernels a coupled step launches: the gather, the particle kernel, the bead
// diagnostics, the lattice pass, the source, and the next step's lists.
long long step_launches(const lbmd_handle *h) { return h->total_beads > 0 ? 6 : 2; }

// the event marking the end of the latest k_lists launch: a separate one
// inside a stream capture
cudaEvent_t lists_event(const lbmd_handle *h) { return h->capturing ? h->ev_lists_cap : h->ev_lists; }

// k_lists for the current bead positions on the particle stream, where the
// next particle kernel follows it; ev_lists marks its end.
lbmd_status enqueue_lists(lbmd_handle *h) {
    {
        ProfScope ps(h, K_LISTS, h->aux);
        CK(launch_lists(h->S, h->aux));
    }
    CK(cudaEventRecord(lists_event(h), h->aux));
    h->lists_ready = true;
    if (h->capturing) h->lists_in_capture = true;
    return LBMD_OK;
}

// Lists for the current positions queued (outside any capture) and joined
// into the main stream: before a graph launch or a capture, whose first step
// relies on them.
lbmd_status lists_before_graph(lbmd_handle *h) {
    if (h->total_beads == 0) return LBMD_OK;
    if (!h->lists_ready) {
        CK(cudaEventRecord(h->ev_pre, h->st));
        CK(cudaStreamWaitEvent(h->aux, h->ev_pre, 0));
        lbmd_status s = enqueue_lists(h);
        if (s != LBMD_OK) return s;
        h->launches += 1;
    }
    CK(cudaStreamWaitEvent(h->st, h->ev_lists, 0));
    return LBMD_OK;
}

lbmd_status enqueue_gather(lbmd_handle *h) {
    if (h->total_beads > 0) {
        // the step's starting Verlet lists: normally queued by the previous
        // step right after its particle kernel, so they overlap its source
        // pass and this gather; else queued here, beside the gather
        if (!h->lists_ready) {
            CK(cudaEventRecord(h->ev_pre, h->st));
            CK(cudaStreamWaitEvent(h->aux, h->ev_pre, 0));
            lbmd_status s = enqueue_lists(h);
            if (s != LBMD_OK) return s;
            h->launches += 1;
        }
        {
            ProfScope ps(h, K_GATHER, h->st);
            CK(launch_gather(h->S, h->popA, h->st));
        }
        // the lattice pass starts no earlier than the particle kernel can: a
        // lattice pass already spread over every SM would keep the particle
        // blocks (each asks for a whole SM's shared memory when reserving)
        // waiting until it drained.  (Inside a capture whose lists were
        // queued before it, the graph launch itself waits for them.)
        if (!h->capturing || h->lists_in_capture) CK(cudaStreamWaitEvent(h->st, lists_event(h), 0));
    }
    return LBMD_OK;
}

lbmd_status enqueue_advance(lbmd_handle *h) {
    CK(cudaEventRecord(h->ev_fork, h->st));
    CK(cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
    {
        ProfScope ps(h, K_PARTICLES, h->aux);
        CK(launch_particles(h->S, h->popA, h->aux));
    }
    CK(cudaEventRecord(h->ev_join, h->aux));
    // the next step's starting lists, from the positions this particle kernel
    // leaves, beside this step's source pass and the next gather
    if (h->total_beads > 0) {
        lbmd_status s = enqueue_lists(h);
        if (s != LBMD_OK) return s;
    }
    if (h->total_beads > 0) {
        CK(cudaStreamWaitEvent(h->aux2, h->ev_fork, 0));
        {
            ProfScope ps(h, K_BEAD_DIAG, h->aux2);
            CK(launch_bead_diag(h->S, h->aux2));
        }
        CK(cudaEventRecord(h->ev_join2, h->aux2));
    }
    if (!h->overlap) CK(cudaStreamWaitEvent(h->st, h->ev_join, 0));
    {
        ProfScope ps(h, K_STREAM_COLLIDE, h->st);
        CK(lattice_pass(h, h->S, h->by, h->zc, true));
    }
    CK(cudaStreamWaitEvent(h->st, h->ev_join, 0));
    if (h->total_beads > 0) CK(cudaStreamWaitEvent(h->st, h->ev_join2, 0));
    {
        ProfScope ps(h, K_SOURCE, h->st);
        CK(launch_source(h->S, h->popB, h->st));
    }
    std::swap(h->popA, h->popB);
    h->host_step += 1;
    h->launches += step_launches(h);
    if (h->pending.size() > 30000) return resolve_profile(h);
    return LBMD_OK;
}

lbmd_status enqueue_step(lbmd_handle *h) {
    lbmd_status s = enqueue_gather(h);
    return s == LBMD_OK ? enqueue_advance(h) : s;
}

lbmd_status slab_only(lbmd_handle *h) {
    if (!h) return LBMD_ERR_INVALID_ARG;
    if (!h->S.slab) return fail(h, LBMD_ERR_INVALID_ARG, "not a slab handle (slab_nx = 0)");
    return LBMD_OK;
}

lbmd_status not_slab(lbmd_handle *h, const char *what) {
    if (h && h->S.slab) return fail(h, LBMD_ERR_INVALID_ARG, std::string(what) + " is not available in slab mode");
    return LBMD_OK;
}

void drop_graph(lbmd_handle *h) {
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
    h->graph_A = nullptr;
    if (h->lexec) cudaGraphExecDestroy(h->lexec);
    h->lexec = nullptr;
    h->loop_A = nullptr;
}

// One tick of the device-side step loop: the body of two steps has run once
// more; the loop goes on while bodies remain.
__global__ void k_loop_tick(cudaGraphConditionalHandle hdl, unsigned int *remaining) {
    const unsigned int r = *remaining - 1u;
    *remaining = r;
    cudaGraphSetConditional(hdl, r > 0u ? 1u : 0u);
}

__global__ void k_set_u32(unsigned int *p, unsigned int v) { *p = v; }

// n Philox4x32-10 draws: in [n][6] = (ctr0..ctr3, key0, key1), out [n][4]
__global__ void k_philox_words(const uint32_t *in, uint32_t *out, long long n) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint32_t *a = in + 6 * k;
    const uint4 x = philox4x32_10(make_uint4(a[0], a[1], a[2], a[3]), make_uint2(a[4], a[5]));
    out[4 * k + 0] = x.x;
    out[4 * k + 1] = x.y;
    out[4 * k + 2] = x.z;
    out[4 * k + 3] = x.w;
}

// the bead-noise normals of beads bead0 .. bead0 + n - 1 (the particle
// kernel's own draw)
__global__ void k_noise_gauss3(unsigned long long seed, uint32_t real, uint32_t bead0, long long n, long long step,
                               uint32_t substep, float *out) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float3 z = gauss3(seed, real, bead0 + (uint32_t)k, step, substep);
    out[3 * k + 0] = z.x;
    out[3 * k + 1] = z.y;
    out[3 * k + 2] = z.z;
}

// restart every realization's translocation record at step origin
__global__ void k_reset_transloc(lbmd_transloc *tl, int n_real, long long origin) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_real) return;
    lbmd_transloc e;
    e.t_origin = origin;
    e.t_first = -1;
    e.t_x = -1;
    e.rg_u_origin = -1.0;
    e.rg_t_x = -1.0;
    e.max_translocated = 0.0;
    tl[r] = e;
}

// Graph holding one conditional WHILE node whose body is two coupled steps
// (A -> B -> A, so the buffers line up again) followed by the tick kernel.
// The condition starts at 1 on every launch, so one launch runs
// 2 * (*loopc) steps for *loopc >= 1.
lbmd_status capture_loop(lbmd_handle *h) {
    if (h->lexec) cudaGraphExecDestroy(h->lexec);
    h->lexec = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphCreate");
    cudaGraphConditionalHandle hdl;
    e = cudaGraphConditionalHandleCreate(&hdl, g, 1u, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(h, e, "cudaGraphConditionalHandleCreate"); }
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hdl;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(h, e, "cudaGraphAddNode(conditional)"); }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    void *A0 = h->popA;
    const long long s0 = h->host_step, l0 = h->launches;
    {   // the body's first step relies on lists queued before the loop starts
        lbmd_status sl = lists_before_graph(h);
        if (sl != LBMD_OK) { cudaGraphDestroy(g); return sl; }
    }
    h->capturing = true;
    h->lists_in_capture = false;
    e = cudaStreamBeginCaptureToGraph(h->st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { h->capturing = false; cudaGraphDestroy(g); return cuda_fail(h, e, "cudaStreamBeginCaptureToGraph"); }
    lbmd_status s = enqueue_step(h);
    if (s == LBMD_OK) s = enqueue_step(h);
    // the next body's lists join the body before its end
    if (s == LBMD_OK && h->total_beads > 0 && cudaStreamWaitEvent(h->st, h->ev_lists_cap, 0) != cudaSuccess) s = LBMD_ERR_CUDA;
    if (s == LBMD_OK) {
        k_loop_tick<<<1, 1, 0, h->st>>>(hdl, (unsigned int *)(h->dbuf + h->L.loopc));
        if (cudaGetLastError() != cudaSuccess) s = LBMD_ERR_CUDA;
    }
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(h->st, &captured);
    h->capturing = false;
    h->lists_in_capture = false;
    h->host_step = s0;
    h->launches = l0;
    if (s != LBMD_OK || e != cudaSuccess) {
        cudaGraphDestroy(g);
        return s != LBMD_OK ? s : cuda_fail(h, e, "cudaStreamEndCapture");
    }
    // the kernels keep the priorities of the streams they were captured on
    // (particle kernel high, bead diagnostics low), as in eager launches
    e = cudaGraphInstantiate(&h->lexec, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { h->lexec = nullptr; return cuda_fail(h, e, "cudaGraphInstantiate(loop)"); }
    h->loop_A = A0;
    return LBMD_OK;
}

lbmd_status capture_graph(lbmd_handle *h) {
    drop_graph(h);
    if (h->graph_steps <= 0) return LBMD_OK;
    cudaGraph_t g = nullptr;
    {   // the graph's first step relies on lists queued before each launch
        lbmd_status sl = lists_before_graph(h);
        if (sl != LBMD_OK) return sl;
    }
    h->capturing = true;
    h->lists_in_capture = false;
    void *A0 = h->popA;
    const long long s0 = h->host_step, l0 = h->launches;
    cudaError_t e = cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { h->capturing = false; return cuda_fail(h, e, "cudaStreamBeginCapture"); }
    lbmd_status s = LBMD_OK;
    for (int k = 0; k < h->graph_steps && s == LBMD_OK; ++k) s = enqueue_step(h);
    // the lists for the step after the graph join the graph before its end
    if (s == LBMD_OK && h->total_beads > 0 && cudaStreamWaitEvent(h->st, h->ev_lists_cap, 0) != cudaSuccess) s = LBMD_ERR_CUDA;
    e = cudaStreamEndCapture(h->st, &g);
    h->capturing = false;
    h->lists_in_capture = false;
    h->host_step = s0;
    h->launches = l0;
    if (s != LBMD_OK) { if (g) cudaGraphDestroy(g); return s; }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->gexec, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { h->gexec = nullptr; return cuda_fail(h, e, "cudaGraphInstantiate"); }
    h->graph_A = A0;
    if (h->popA != A0) return fail(h, LBMD_ERR_INVALID_ARG, "graph must hold an even number of steps");
    return LBMD_OK;
}

void build_geometry(const lbmd_config *c, const uint8_t *solid, int near_radius, std::vector<uint32_t> &link,
                    std::vector<unsigned long long> &wallmask, std::vector<uint8_t> &tile,
                    std::vector<uint8_t> &sol, double &n_fluid) {
    const int nx = c->nx, ny = c->ny, nz = c->nz;
    const size_t ns = (size_t)nx * ny * nz;
    sol.assign(solid, solid + ns);
    for (auto &b : sol) b = b ? 1 : 0;
    link.assign(ns, 0u);
    n_fluid = 0;
    static const int C[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
                                 {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
                                 {-1, 0, 1}, {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const size_t s = x + (size_t)nx * (y + (size_t)ny * z);
                if (sol[s]) { link[s] = SOLID_BIT; continue; }
                n_fluid += 1;
                uint32_t m = 0;
                for (int i = 1; i < 19; ++i) {
                    const int sx = (x - C[i][0] + nx) % nx, sy = (y - C[i][1] + ny) % ny, sz = (z - C[i][2] + nz) % nz;
                    if (sol[sx + (size_t)nx * (sy + (size_t)ny * sz)]) m |= 1u << i;
                }
                link[s] = m;
            }
    // near-solid bit: the solid mask dilated by near_radius in the Chebyshev
    // metric, as three separable 1-D maximum filters
    std::vector<uint8_t> a(sol), t(ns);
    const int dims[3] = {nx, ny, nz};
    const size_t stride[3] = {1, (size_t)nx, (size_t)nx * ny};
    for (int ax = 0; ax < 3; ++ax) {
        const int n = dims[ax];
        for (size_t s = 0; s < ns; ++s) {
            const int coord = (int)((s / stride[ax]) % n);
            uint8_t v = 0;
            for (int d = -near_radius; d <= near_radius && !v; ++d) {
                const int q = ((coord + d) % n + n) % n;
                v = a[s + (size_t)(q - coord) * stride[ax]];
            }
            t[s] = v;
        }
        a.swap(t);
    }
    for (size_t s = 0; s < ns; ++s)
        if (a[s]) link[s] |= NEAR_SOLID_BIT;
    // solid sites of the 4x4x4 box [x-1, x+2] x [y-1, y+2] x [z-1, z+2]
    wallmask.assign(ns, 0ull);
    std::vector<int> wx(4 * (size_t)nx), wy(4 * (size_t)ny), wz(4 * (size_t)nz);
    for (int d = 0; d < 4; ++d) {
        for (int i = 0; i < nx; ++i) wx[d * (size_t)nx + i] = ((i + d - 1) % nx + nx) % nx;
        for (int i = 0; i < ny; ++i) wy[d * (size_t)ny + i] = ((i + d - 1) % ny + ny) % ny;
        for (int i = 0; i < nz; ++i) wz[d * (size_t)nz + i] = ((i + d - 1) % nz + nz) % nz;
    }
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                unsigned long long m = 0;
                for (int dz = 0; dz < 4; ++dz)
                    for (int dy = 0; dy < 4; ++dy) {
                        const size_t row = (size_t)nx * (wy[dy * (size_t)ny + y] + (size_t)ny * wz[dz * (size_t)nz + z]);
                        for (int dx = 0; dx < 4; ++dx)
                            if (sol[row + wx[dx * (size_t)nx + x]]) m |= 1ull << (dx + 4 * dy + 16 * dz);
                    }
                wallmask[x + (size_t)nx * (y + (size_t)ny * z)] = m;
            }
    const int nxt = (nx + 31) / 32;
    tile.assign((size_t)nxt * ny * nz, 0);
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                if (link[x + (size_t)nx * (y + (size_t)ny * z)] & ~NEAR_SOLID_BIT)
                    tile[x / 32 + (size_t)nxt * (y + (size_t)ny * z)] = 1;
}

}  // namespace

extern "C" {

const char *lbmd_status_string(lbmd_status s) {
    switch (s) {
        case LBMD_OK: return "ok";
        case LBMD_ERR_INVALID_ARG: return "invalid argument";
        case LBMD_ERR_CUDA: return "CUDA error";
        case LBMD_ERR_NONFINITE: return "non-finite value in the state";
        case LBMD_ERR_TIMEOUT: return "bounded wait timed out";
        case LBMD_ERR_CAPACITY: return "fixed-capacity list overflowed";
        case LBMD_ERR_BUFFER: return "device buffer too small or misaligned";
    }
    return "unknown status";
}

const char *lbmd_last_error(const lbmd_handle *h) { return h ? h->err.c_str() : "null handle"; }

lbmd_status lbmd_philox4x32_10(const uint32_t *ctr_key, uint32_t *out, int64_t n, void *stream) {
    if (n < 0 || (n > 0 && (!ctr_key || !out))) return LBMD_ERR_INVALID_ARG;
    if (n == 0) return LBMD_OK;
    const int threads = 256;
    k_philox_words<<<(unsigned)((n + threads - 1) / threads), threads, 0, (cudaStream_t)stream>>>(ctr_key, out, n);
    return cudaGetLastError() == cudaSuccess ? LBMD_OK : LBMD_ERR_CUDA;
}

lbmd_status lbmd_noise_gauss3(uint64_t seed, uint32_t realization, uint32_t bead0, int64_t n, int64_t step,
                              uint32_t substep, float *out, void *stream) {
    if (n < 0 || (n > 0 && !out) || (double)bead0 + (double)n > 4294967296.0) return LBMD_ERR_INVALID_ARG;
    if (n == 0) return LBMD_OK;
    const int threads = 256;
    k_noise_gauss3<<<(unsigned)((n + threads - 1) / threads), threads, 0, (cudaStream_t)stream>>>(
        (unsigned long long)seed, realization, bead0, n, step, substep, out);
    return cudaGetLastError() == cudaSuccess ? LBMD_OK : LBMD_ERR_CUDA;
}

lbmd_status lbmd_required_bytes(const lbmd_config *cfg, const int32_t *bead_offsets, size_t *bytes) {
    std::string why;
    if (!bytes || !config_ok(cfg, bead_offsets, why)) return LBMD_ERR_INVALID_ARG;
    *bytes = layout_of(cfg, bead_offsets[cfg->n_real]).total;
    return LBMD_OK;
}

lbmd_status lbmd_init(const lbmd_config *cfg, const uint8_t *solid, const int32_t *bead_offsets, const double *r_init,
                      void *device_buffer, size_t device_bytes, void *stream, lbmd_handle **out) {
    if (!out) return LBMD_ERR_INVALID_ARG;
    *out = nullptr;
    cudaGetLastError();  // an error the caller left pending is not this handle's
    std::string why;
    if (!config_ok(cfg, bead_offsets, why) || !solid) return LBMD_ERR_INVALID_ARG;
    lbmd_handle *h = new lbmd_handle();
    h->cfg = *cfg;
    h->offsets.assign(bead_offsets, bead_offsets + cfg->n_real + 1);
    h->total_beads = bead_offsets[cfg->n_real];
    if (h->total_beads > 0 && !r_init) { delete h; return LBMD_ERR_INVALID_ARG; }
    h->L = layout_of(cfg, h->total_beads);
    if (!device_buffer || ((uintptr_t)device_buffer & 255u) || device_bytes < h->L.total) {
        delete h;
        return LBMD_ERR_BUFFER;
    }
    h->dbuf = (char *)device_buffer;
    h->dbytes = device_bytes;
    h->st = (cudaStream_t)stream;
    auto bail = [&](lbmd_status s) { lbmd_destroy(h); return s; };
    {
        int lo = 0, hi = 0;
        cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->aux, cudaStreamNonBlocking, hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->aux2, cudaStreamNonBlocking, lo);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join2, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_pre, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_lists, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_lists_cap, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->bst, cudaStreamNonBlocking, hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->baux, cudaStreamNonBlocking, hi);
        cudaEvent_t *bev[] = {&h->ev_bfork, &h->ev_bjoin, &h->ev_bstart, &h->ev_rep[0], &h->ev_rep[1], &h->ev_bwd[0],
                              &h->ev_bwd[1]};
        for (cudaEvent_t *ev : bev)
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        if (e != cudaSuccess) { cuda_fail(h, e, "stream/event creation"); return bail(LBMD_ERR_CUDA); }
    }
    const Layout &L = h->L;
    char *b = h->dbuf;
    h->popA = b + L.popA;
    h->popB = b + L.popB;
    h->staging = (float *)(b + L.staging);

    // geometry on the host
    std::vector<uint32_t> link;
    std::vector<unsigned long long> wallmask;
    std::vector<uint8_t> tile, sol;
    double n_fluid = 0;
    // a bead's wall-list box reaches floor(rlw) + 1 sites from its cell corner
    const int near_radius = (int)std::floor(std::pow(2.0, 1.0 / 6.0) * cfg->wall_sigma + 0.5 * SKIN) + 1;
    const bool slab = cfg->slab_nx > 0;
    const int nxl = local_nx(cfg);
    std::vector<uint32_t> glink;
    std::vector<unsigned long long> gwallmask;
    if (slab) {
        // the slab's planes with their ghosts, cut from the whole lattice's
        // mask (periodic in x); the link words of the two outermost ghost
        // planes see the other edge and are never used.  The beads keep the
        // whole lattice's geometry for their wall lists.
        lbmd_config lcfg = *cfg;
        lcfg.nx = nxl;
        std::vector<uint8_t> lsol((size_t)nxl * cfg->ny * cfg->nz);
        for (int z = 0; z < cfg->nz; ++z)
            for (int y = 0; y < cfg->ny; ++y)
                for (int xl = 0; xl < nxl; ++xl) {
                    const int xg = ((cfg->slab_x0 - 1 + xl) % cfg->nx + cfg->nx) % cfg->nx;
                    lsol[xl + (size_t)nxl * (y + (size_t)cfg->ny * z)] = solid[xg + (size_t)cfg->nx * (y + (size_t)cfg->ny * z)];
                }
        double nf_local = 0;
        build_geometry(&lcfg, lsol.data(), near_radius, link, wallmask, tile, sol, nf_local);
        std::vector<uint8_t> gtile, gsol;
        double nf_all = 0;
        build_geometry(cfg, solid, near_radius, glink, gwallmask, gtile, gsol, nf_all);
        for (int z = 0; z < cfg->nz; ++z)  // fluid sites of the slab's own planes
            for (int y = 0; y < cfg->ny; ++y)
                for (int xl = 1; xl <= cfg->slab_nx; ++xl)
                    n_fluid += sol[xl + (size_t)nxl * (y + (size_t)cfg->ny * z)] ? 0.0 : 1.0;
    } else {
        build_geometry(cfg, solid, near_radius, link, wallmask, tile, sol, n_fluid);
    }

    Sim &S = h->S;
    memset(&S, 0, sizeof(S));
    S.nx = nxl; S.ny = cfg->ny; S.nz = cfg->nz;
    S.ns = nxl * cfg->ny * cfg->nz;
    S.ps = (int)pop_stride((size_t)S.ns);
    S.nxt = (nxl + 31) / 32;
    S.inx = 1.0f / (float)nxl;
    S.slab = slab ? 1 : 0;
    S.bnx = cfg->nx;
    S.binx = 1.0f / (float)cfg->nx;
    S.gx0 = slab ? ((cfg->slab_x0 - 1) % cfg->nx + cfg->nx) % cfg->nx : 0;
    S.own_lo = slab ? 1 : 0;
    S.own_hi = slab ? cfg->slab_nx + 1 : nxl;
    S.iny = 1.0f / (float)cfg->ny;
    S.inz = 1.0f / (float)cfg->nz;
    S.n_real = cfg->n_real;
    S.real_base = (uint32_t)cfg->real_base;
    S.interp = cfg->interp;
    S.integrator = cfg->integrator;
    S.fluct = cfg->lb_kT > 0.0;
    {   // fluctuating LB: mode k gets variance mu b_k (1 - gamma^2), mu = rho kT / c_s^2,
        // gamma = 1 - omega; per unit sqrt(rho) and weight: sqrt(3 kT (1 - gamma^2) / b_k)
        const double gam = 1.0 - 1.0 / cfg->tau;
        for (int k = 4; k < LBMD_Q; ++k) {
            double b = 0.0;
            for (int i = 0; i < LBMD_Q; ++i) b += wq_exact(i) * (double)mode_e(k, i) * (double)mode_e(k, i);
            S.fl_amp[k - 4] = (float)std::sqrt(3.0 * cfg->lb_kT * (1.0 - gam * gam) / b);
        }
    }
    {   // stochastic position Verlet constants over one sub-step h (double, then stored)
        const double hsub = 1.0 / cfg->md_outer / cfg->md_inner;
        const double c1 = std::exp(-cfg->gamma * hsub);
        S.spv_c = (float)c1;
        S.spv_g1 = (float)(cfg->gamma > 0.0 ? (1.0 - c1) / cfg->gamma : hsub);
        S.spv_sig = (float)(cfg->kT > 0.0 ? std::sqrt(cfg->kT * (1.0 - c1 * c1)) : 0.0);
    }
    S.precision = cfg->precision;
    S.omega = (float)(1.0 / cfg->tau);
    for (int a = 0; a < 3; ++a) S.g[a] = (float)cfg->body_force[a];
    S.n_fluid = n_fluid;
    S.total_beads = h->total_beads;
    int maxb = 0;
    for (int r = 0; r < cfg->n_real; ++r) maxb = std::max(maxb, bead_offsets[r + 1] - bead_offsets[r]);
    S.max_beads = maxb;
    S.wall_x = cfg->wall_x;
    S.pore_h = cfg->pore_h;
    S.pore_ylo = cfg->ny / 2 - cfg->pore_h / 2;
    S.pore_zlo = cfg->nz / 2 - cfg->pore_h / 2;
    S.k_bond = (float)cfg->k_bond;
    S.r0 = (float)cfg->r0;
    S.kappa = (float)cfg->kappa_bend;
    const double c13 = std::pow(2.0, 1.0 / 3.0), c16 = std::pow(2.0, 1.0 / 6.0);
    S.lj_eps = (float)cfg->lj_eps;
    S.lj_sig2 = (float)(cfg->lj_sigma * cfg->lj_sigma);
    S.lj_rc2 = (float)(c13 * cfg->lj_sigma * cfg->lj_sigma);
    S.wall_eps = (float)cfg->wall_eps;
    S.wall_sig2 = (float)(cfg->wall_sigma * cfg->wall_sigma);
    S.wall_rc2 = (float)(c13 * cfg->wall_sigma * cfg->wall_sigma);
    S.E = (float)cfg->E;
    S.gamma = (float)cfg->gamma;
    S.kT = (float)cfg->kT;
    S.M = cfg->md_outer;
    S.Mb = cfg->md_inner;
    S.skin_half2 = (float)(0.25 * SKIN * SKIN);
    // bead pairs: both beads may move skin/2; solid sites do not move, so the
    // wall list needs only the cut-off plus the bead's own skin/2
    const double rl = c16 * cfg->lj_sigma + SKIN, rlw = c16 * cfg->wall_sigma + 0.5 * SKIN;
    S.rl2 = (float)(rl * rl);
    S.rlw = (float)rlw;
    S.rlw2 = (float)(rlw * rlw);
    const int dims[3] = {cfg->nx, cfg->ny, cfg->nz};
    for (int a = 0; a < 3; ++a) {
        S.ncell[a] = std::max(1, (int)std::floor(dims[a] / rl));
        S.cell_per_site[a] = (float)S.ncell[a] / (float)dims[a];
    }
    S.wallmask = (const unsigned long long *)(b + L.wallmask);
    S.seed = cfg->seed;
    S.link = (const uint32_t *)(b + L.link);
    S.blink = slab ? (const uint32_t *)(b + L.blink) : S.link;
    S.bwallmask = slab ? (const unsigned long long *)(b + L.bwallmask) : S.wallmask;
    S.tileflag = (const uint8_t *)(b + L.tileflag);
    S.solid = (const uint8_t *)(b + L.solid);
    S.G = (unsigned long long *)(b + L.G);
    S.stamp = (int *)(b + L.stamp);
    S.r_hi = (float4 *)(b + L.r_hi);
    S.r_lo = (float4 *)(b + L.r_lo);
    S.v = (float4 *)(b + L.v);
    S.up = (float4 *)(b + L.up);
    S.J = (float4 *)(b + L.J);
    S.pair_node = (int *)(b + L.pair_node);
    S.pair_w = (float *)(b + L.pair_w);
    S.bead_real = (const int *)(b + L.bead_real);
    S.bead_off = (const int *)(b + L.bead_off);
    S.bsnap = (float4 *)(b + L.bsnap);
    S.md_map = (const int4 *)(b + L.md_map);
    S.nbr_g = (uint16_t *)(b + L.nbr_g);
    S.wal_g = (uint32_t *)(b + L.wal_g);
    S.nn_g = (int *)(b + L.nn_g);
    S.nw_g = (int *)(b + L.nw_g);
    S.md_clusters = 0;
    S.fsum = (long long *)(b + L.fsum);
    S.ring = (lbmd_diag *)(b + L.ring);
    S.obs = (lbmd_obs *)(b + L.obs);
    S.tl = (lbmd_transloc *)(b + L.tl);
    S.ctrl = (Ctrl *)(b + L.ctrl);
    S.phase = nullptr;
    {
        int dev = 0, optin = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess)
            S.smem_optin = optin;
    }

#define CKI(call)                                                           \
    do {                                                                    \
        cudaError_t e__ = (call);                                           \
        if (e__ != cudaSuccess) { cuda_fail(h, e__, #call); return bail(LBMD_ERR_CUDA); } \
    } while (0)
    CKI(cudaMemcpyAsync(b + L.link, link.data(), link.size() * 4, cudaMemcpyHostToDevice, h->st));
    CKI(cudaMemcpyAsync(b + L.wallmask, wallmask.data(), wallmask.size() * 8, cudaMemcpyHostToDevice, h->st));
    CKI(cudaMemcpyAsync(b + L.tileflag, tile.data(), tile.size(), cudaMemcpyHostToDevice, h->st));
    CKI(cudaMemcpyAsync(b + L.solid, sol.data(), sol.size(), cudaMemcpyHostToDevice, h->st));
    if (slab) {
        CKI(cudaMemcpyAsync(b + L.blink, glink.data(), glink.size() * 4, cudaMemcpyHostToDevice, h->st));
        CKI(cudaMemcpyAsync(b + L.bwallmask, gwallmask.data(), gwallmask.size() * 8, cudaMemcpyHostToDevice, h->st));
    }
    CKI(cudaMemcpyAsync(b + L.bead_off, h->offsets.data(), h->offsets.size() * 4, cudaMemcpyHostToDevice, h->st));
    std::vector<int32_t> breal((size_t)std::max(h->total_beads, 1), 0);
    for (int r = 0; r < cfg->n_real; ++r)
        for (int i = bead_offsets[r]; i < bead_offsets[r + 1]; ++i) breal[i] = r;
    CKI(cudaMemcpyAsync(b + L.bead_real, breal.data(), breal.size() * 4, cudaMemcpyHostToDevice, h->st));
    CKI(cudaStreamSynchronize(h->st));
    CKI(cudaMemsetAsync(b + L.G, 0, (size_t)cfg->n_real * 3 * S.ns * 8, h->st));
    CKI(cudaMemsetAsync(b + L.stamp, 0, (size_t)cfg->n_real * S.ns * 4, h->st));
    CKI(cudaMemsetAsync(b + L.ring, 0, (size_t)cfg->n_real * LBMD_DIAG_RING * sizeof(lbmd_diag), h->st));
    CKI(cudaMemsetAsync(b + L.obs, 0, (size_t)cfg->n_real * sizeof(lbmd_obs), h->st));
    CKI(cudaMemsetAsync(b + L.ctrl, 0, sizeof(Ctrl), h->st));
    CKI(cudaMemsetAsync(b + L.fsum, 0, (size_t)cfg->n_real * 8 * sizeof(long long), h->st));
    CKI(cudaMemsetAsync(b + L.popB, 0, L.staging - L.popB, h->st));
    CKI(cudaMemsetAsync(b + L.up, 0, (size_t)std::max(h->total_beads, 1) * 32, h->st));
    CKI(launch_init_rest(S, h->popA, h->st));
    CKI(cudaStreamSynchronize(h->st));
    encode_tensor_maps(h);
    // the particle kernel needs its shared-memory size granted once
    if (md_shape(S).smem > 200 * 1024) { fail(h, LBMD_ERR_CAPACITY, "too many beads per realization for shared memory"); return bail(LBMD_ERR_CAPACITY); }
    lbmd_status s = lbmd_set_beads(h, r_init, nullptr);
    if (s == LBMD_OK) s = lbmd_reset_translocation(h);
    if (s == LBMD_OK) s = upload_md_map(h, h->S, 0);
    if (s == LBMD_OK) s = cudaStreamSynchronize(h->st) == cudaSuccess ? LBMD_OK : LBMD_ERR_CUDA;
    if (s != LBMD_OK) return bail(s);
    *out = h;
    return LBMD_OK;
#undef CKI
}

lbmd_status lbmd_step(lbmd_handle *h, int64_t n) {
    if (!h || n < 0) return LBMD_ERR_INVALID_ARG;
    if (not_slab(h, "lbmd_step") != LBMD_OK) return LBMD_ERR_INVALID_ARG;
    while (n > 0) {
        const bool use_graph = h->graph_steps > 0 && !h->profiling && n >= h->graph_steps;
        if (use_graph) {
            if (!h->gexec) {
                lbmd_status s = capture_graph(h);
                if (s != LBMD_OK) return s;
            }
            if (h->popA == h->graph_A) {
                lbmd_status sl = lists_before_graph(h);
                if (sl != LBMD_OK) return sl;
                CK(cudaGraphLaunch(h->gexec, h->st));
                h->lists_ready = h->total_beads > 0;  // the graph's last step queued the next lists
                h->host_step += h->graph_steps;
                h->launches += step_launches(h) * h->graph_steps;
                n -= h->graph_steps;
                continue;
            }
        }
        lbmd_status s = enqueue_step(h);
        if (s != LBMD_OK) return s;
        n -= 1;
    }
    return LBMD_OK;
}

lbmd_status lbmd_step_loop(lbmd_handle *h, int64_t n) {
    if (!h || n < 0) return LBMD_ERR_INVALID_ARG;
    if (not_slab(h, "lbmd_step_loop") != LBMD_OK) return LBMD_ERR_INVALID_ARG;
    if (!h->st) return fail(h, LBMD_ERR_INVALID_ARG, "graph capture needs a non-default stream");
    if (h->profiling) return lbmd_step(h, n);
    if (h->lexec && h->popA != h->loop_A && n > 0) {  // realign A with the captured body
        lbmd_status s = enqueue_step(h);
        if (s != LBMD_OK) return s;
        n -= 1;
    }
    const int64_t pairs = n / 2;
    if (pairs >= 1) {
        if (pairs > 0xffffffffll) return fail(h, LBMD_ERR_INVALID_ARG, "too many steps for one loop launch");
        if (!h->lexec) {
            lbmd_status s = capture_loop(h);
            if (s != LBMD_OK) return s;
        }
        lbmd_status sl = lists_before_graph(h);
        if (sl != LBMD_OK) return sl;
        k_set_u32<<<1, 1, 0, h->st>>>((unsigned int *)(h->dbuf + h->L.loopc), (unsigned int)pairs);
        CK(cudaGetLastError());
        CK(cudaGraphLaunch(h->lexec, h->st));
        h->lists_ready = h->total_beads > 0;  // the loop's last step queued the next lists
        h->host_step += 2 * pairs;
        h->launches += 1 + (2LL * step_launches(h) + 1) * pairs;
    }
    if (n & 1) return enqueue_step(h);
    return LBMD_OK;
}

lbmd_status lbmd_check(lbmd_handle *h) {
    if (!h) return LBMD_ERR_INVALID_ARG;
    Ctrl c;
    CK(cudaMemcpyAsync(&c, h->S.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (c.status & ST_NONFINITE) return fail(h, LBMD_ERR_NONFINITE, "non-finite value in the fluid or bead state");
    if (c.status & ST_CAPACITY) return fail(h, LBMD_ERR_CAPACITY, "neighbour or wall list overflowed");
    if (c.status & ST_TIMEOUT) return fail(h, LBMD_ERR_TIMEOUT, "a bounded device wait gave up");
    return LBMD_OK;
}

lbmd_status lbmd_observables(lbmd_handle *h, lbmd_obs *out) {
    if (!h || !out) return LBMD_ERR_INVALID_ARG;
    if (not_slab(h, "lbmd_observables") != LBMD_OK) return LBMD_ERR_INVALID_ARG;
    CK(launch_fluid_observables(h->S, h->popA, h->st));
    CK(launch_bead_observables(h->S, h->popA, h->st));
    h->launches += 2;
    Ctrl c;
    CK(cudaMemcpyAsync(out, h->S.obs, sizeof(lbmd_obs) * h->cfg.n_real, cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(&c, h->S.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    int st = LBMD_OK;
    if (c.status & ST_NONFINITE) st = LBMD_ERR_NONFINITE;
    else if (c.status & ST_CAPACITY) st = LBMD_ERR_CAPACITY;
    else if (c.status & ST_TIMEOUT) st = LBMD_ERR_TIMEOUT;
    for (int r = 0; r < h->cfg.n_real; ++r) {
        out[r].step = c.step;
        out[r].status = st;
    }
    return LBMD_OK;
}

lbmd_status lbmd_diagnostics(lbmd_handle *h, lbmd_diag *out, int32_t max_rows, int32_t *rows) {
    if (!h || !out || !rows || max_rows < 0) return LBMD_ERR_INVALID_ARG;
    const int R = h->cfg.n_real;
    const long long done = h->host_step;  // rows exist for steps [0, done)
    const long long avail = std::min<long long>(done, LBMD_DIAG_RING);
    const int n = (int)std::min<long long>(avail, max_rows);
    // only the rows returned cross to the host: the ring slots of steps
    // [done - n, done), at most two runs per realization (the ring wraps),
    // each one strided copy over the realizations
    const size_t row = sizeof(lbmd_diag);
    const int s0 = (int)((done - n) % LBMD_DIAG_RING);
    const int first = std::min(n, LBMD_DIAG_RING - s0);
    if (first > 0)
        CK(cudaMemcpy2DAsync(out, (size_t)max_rows * row, h->S.ring + s0, (size_t)LBMD_DIAG_RING * row, (size_t)first * row, R,
                             cudaMemcpyDeviceToHost, h->st));
    if (n > first)
        CK(cudaMemcpy2DAsync(out + first, (size_t)max_rows * row, h->S.ring, (size_t)LBMD_DIAG_RING * row,
                             (size_t)(n - first) * row, R, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    *rows = n;
    return LBMD_OK;
}

lbmd_status lbmd_translocation(lbmd_handle *h, lbmd_transloc *out) {
    if (!h || !out) return LBMD_ERR_INVALID_ARG;
    CK(cudaMemcpyAsync(out, h->S.tl, (size_t)h->cfg.n_real * sizeof(lbmd_transloc), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    return LBMD_OK;
}

lbmd_status lbmd_reset_translocation(lbmd_handle *h) {
    if (!h) return LBMD_ERR_INVALID_ARG;
    const int R = h->cfg.n_real;
    k_reset_transloc<<<(R + 127) / 128, 128, 0, h->st>>>(h->S.tl, R, (long long)h->host_step);
    CK(cudaGetLastError());
    h->launches += 1;
    return LBMD_OK;
}

lbmd_status lbmd_init_fluid(lbmd_handle *h, const double *rho, const double *u) {
    if (!h) return LBMD_ERR_INVALID_ARG;
    const size_t ns = h->S.ns;
    std::vector<float> rows(4 * ns);
    for (int r = 0; r < h->cfg.n_real; ++r) {
        for (size_t s = 0; s < ns; ++s) {
            rows[s] = rho ? (float)rho[(size_t)r * ns + s] : 1.0f;
            for (int a = 0; a < 3; ++a) rows[(a + 1) * ns + s] = u ? (float)u[((size_t)r * 3 + a) * ns + s] : 0.0f;
        }
        CK(cudaMemcpyAsync(h->staging + ((size_t)r * LBMD_Q + 15) * ns, rows.data(), 4 * ns * sizeof(float),
                           cudaMemcpyHostToDevice, h->st));
        CK(cudaStreamSynchronize(h->st));
    }
    CK(launch_feq_to_staging(h->S, h->staging, h->st));
    CK(launch_push_from_staging(h->S, h->staging, h->popA, true, h->st));
    h->launches += 2;
    CK(cudaStreamSynchronize(h->st));
    return LBMD_OK;
}

static lbmd_status pull_out(lbmd_handle *h, float *f, bool dev) {
    if (!h || !f) return LBMD_ERR_INVALID_ARG;
    CK(launch_pull_to_staging(h->S, h->popA, h->staging, dev, h->st));
    h->launches += 1;
    CK(cudaMemcpyAsync(f, h->staging, (size_t)h->cfg.n_real * LBMD_Q * h->S.ns * sizeof(float),
                       cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    return LBMD_OK;
}

lbmd_status lbmd_get_populations(lbmd_handle *h, float *f) { return pull_out(h, f, false); }

lbmd_status lbmd_get_deviations(lbmd_handle *h, float *dev) { return pull_out(h, dev, true); }

static lbmd_status push_in(lbmd_handle *h, const float *f, bool dev) {
    if (!h || !f) return LBMD_ERR_INVALID_ARG;
    CK(cudaMemcpyAsync(h->staging, f, (size_t)h->cfg.n_real * LBMD_Q * h->S.ns * sizeof(float),
                       cudaMemcpyHostToDevice, h->st));
    CK(launch_push_from_staging(h->S, h->staging, h->popA, dev, h->st));
    h->launches += 1;
    CK(cudaStreamSynchronize(h->st));
    return LBMD_OK;
}

lbmd_status lbmd_set_populations(lbmd_handle *h, const float *f) { return push_in(h, f, false); }

lbmd_status lbmd_set_deviations(lbmd_handle *h, const float *dev) { return push_in(h, dev, true); }

lbmd_status lbmd_get_beads(lbmd_handle *h, double *r, double *v) {
    if (!h) return LBMD_ERR_INVALID_ARG;
    const int n = h->total_beads;
    if (n == 0) return LBMD_OK;
    std::vector<float4> hi(n), lo(n), vv(n);
    CK(cudaMemcpyAsync(hi.data(), h->S.r_hi, n * 16, cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(lo.data(), h->S.r_lo, n * 16, cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(vv.data(), h->S.v, n * 16, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    for (int i = 0; i < n; ++i) {
        if (r) {
            r[3 * i] = (double)hi[i].x + (double)lo[i].x;
            r[3 * i + 1] = (double)hi[i].y + (double)lo[i].y;
            r[3 * i + 2] = (double)hi[i].z + (double)lo[i].z;
        }
        if (v) { v[3 * i] = vv[i].x; v[3 * i + 1] = vv[i].y; v[3 * i + 2] = vv[i].z; }
    }
    return LBMD_OK;
}

lbmd_status lbmd_set_beads(lbmd_handle *h, const double *r, const double *v) {
    if (!h) return LBMD_ERR_INVALID_ARG;
    const int n = h->total_beads;
    if (n == 0) return LBMD_OK;
    if (!r) return LBMD_ERR_INVALID_ARG;
    std::vector<float4> hi(n), lo(n), vv(n);
    for (int i = 0; i < n; ++i) {
        float t[3], l[3];
        for (int a = 0; a < 3; ++a) {
            t[a] = (float)r[3 * i + a];
            l[a] = (float)(r[3 * i + a] - (double)t[a]);
        }
        hi[i] = make_float4(t[0], t[1], t[2], 0.f);
        lo[i] = make_float4(l[0], l[1], l[2], 0.f);
        vv[i] = v ? make_float4((float)v[3 * i], (float)v[3 * i + 1], (float)v[3 * i + 2], 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    h->lists_ready = false;  // the next particle kernel needs lists of these positions
    CK(cudaMemcpyAsync(h->S.r_hi, hi.data(), n * 16, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(h->S.r_lo, lo.data(), n * 16, cudaMemcpyHostToDevice, h->st));
    CK(cudaMemcpyAsync(h->S.v, vv.data(), n * 16, cudaMemcpyHostToDevice, h->st));
    CK(cudaStreamSynchronize(h->st));
    return LBMD_OK;
}

lbmd_status lbmd_get_coupling(lbmd_handle *h, float *up, float *J) {
    if (!h) return LBMD_ERR_INVALID_ARG;
    const int n = h->total_beads;
    if (n == 0) return LBMD_OK;
    std::vector<float4> a(n), b(n);
    CK(cudaMemcpyAsync(a.data(), h->S.up, n * 16, cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(b.data(), h->S.J, n * 16, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    for (int i = 0; i < n; ++i) {
        if (up) { up[3 * i] = a[i].x; up[3 * i + 1] = a[i].y; up[3 * i + 2] = a[i].z; }
        if (J) { J[3 * i] = b[i].x; J[3 * i + 1] = b[i].y; J[3 * i + 2] = b[i].z; }
    }
    return LBMD_OK;
}

lbmd_status lbmd_get_step(lbmd_handle *h, int64_t *step) {
    if (!h || !step) return LBMD_ERR_INVALID_ARG;
    *step = h->host_step;
    return LBMD_OK;
}

lbmd_status lbmd_set_step(lbmd_handle *h, int64_t step) {
    if (!h || step < 0) return LBMD_ERR_INVALID_ARG;
    long long s = step;
    CK(cudaMemcpyAsync(&h->S.ctrl->step, &s, sizeof(s), cudaMemcpyHostToDevice, h->st));
    // the source marks the sites it has served with a tag made from the step
    // number; after a jump of the counter an old mark could carry the tag of
    // a coming step, so the marks are cleared
    CK(cudaMemsetAsync(h->S.stamp, 0, (size_t)h->cfg.n_real * h->S.ns * sizeof(int), h->st));
    CK(cudaStreamSynchronize(h->st));
    h->host_step = step;
    return LBMD_OK;
}

lbmd_status lbmd_set_drive(lbmd_handle *h, double gamma, double E) {
    if (!h || !(gamma >= 0.0) || !std::isfinite(gamma) || !std::isfinite(E))
        return fail(h, LBMD_ERR_INVALID_ARG, "gamma must be finite and >= 0, E finite");
    h->cfg.gamma = gamma;
    h->cfg.E = E;
    h->S.gamma = (float)gamma;
    h->S.E = (float)E;
    const double hsub = 1.0 / h->cfg.md_outer / h->cfg.md_inner;
    const double c1 = std::exp(-gamma * hsub);
    h->S.spv_c = (float)c1;
    h->S.spv_g1 = (float)(gamma > 0.0 ? (1.0 - c1) / gamma : hsub);
    h->S.spv_sig = (float)(h->cfg.kT > 0.0 ? std::sqrt(h->cfg.kT * (1.0 - c1 * c1)) : 0.0);
    drop_graph(h);  // the graph holds the old parameters in its kernel arguments
    return LBMD_OK;
}

// ---------------------------------------------------------------------------
// reverse mode
// ---------------------------------------------------------------------------
namespace {

struct AdjLayout {
    size_t pop, bead, traj;      // bytes of one population set, bead state (hi, lo, v), trajectory record
    size_t ck_rec, seg_rec;      // bytes of one checkpoint, one replayed step
    int nck, nseg;               // checkpoints (+ the final state), steps per segment
    size_t ck, seg, lamA, lamB, lam_r, lam_v, LU, adj_node, dpar, stamp, total;
};

AdjLayout adj_layout(const lbmd_handle *h, int K, int C) {
    AdjLayout a;
    const Sim &S = h->S;
    const size_t TB = (size_t)std::max(h->total_beads, 1);
    a.pop = (size_t)h->cfg.n_real * LBMD_Q * S.ps * sizeof(float);
    a.bead = 3 * TB * 16;
    a.traj = (size_t)traj_slots(S.M, S.Mb) * TB * 16;
    a.ck_rec = align256(a.pop) + align256(a.bead);
    a.seg_rec = align256(a.pop) + align256(a.traj);
    a.nck = (K + C - 1) / C + 1;
    a.nseg = std::min(C, K);
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
    a.ck = take(a.ck_rec * a.nck);
    a.seg = take(2 * a.seg_rec * a.nseg);  // two segments: one replayed while the other runs backward
    a.lamA = take(a.pop);
    a.lamB = take(a.pop);
    a.lam_r = take(TB * 16);
    a.lam_v = take(TB * 16);
    a.LU = take((size_t)h->cfg.n_real * 3 * S.ns * 8);
    a.adj_node = take(TB * 8 * 4);
    a.dpar = take((size_t)h->cfg.n_real * 2 * sizeof(double));
    a.stamp = take((size_t)h->cfg.n_real * S.ns * sizeof(int));
    a.total = o;
    return a;
}

bool adjoint_ok(const lbmd_handle *h, int K, int C, std::string &why) {
    if (h->cfg.precision != LBMD_FP32) { why = "the adjoint needs FP32 populations"; return false; }
    if (h->cfg.integrator != 0) { why = "the adjoint follows the velocity-Verlet cycle (integrator 0)"; return false; }
    if (h->cfg.lb_kT != 0.0) { why = "the adjoint needs a deterministic fluid (lb_kT = 0)"; return false; }
    if (K < 1 || C < 1) { why = "K and checkpoint_every must be >= 1"; return false; }
    for (int r = 0; r < h->cfg.n_real; ++r)
        if (h->offsets[r + 1] <= h->offsets[r]) { why = "every realization needs at least one bead"; return false; }
    if (std::pow(2.0, 1.0 / 6.0) * h->cfg.wall_sigma >= 2.0) { why = "bead-wall cut-off must be below 2"; return false; }
    if (h->cfg.kT > 0.0 && !(h->cfg.gamma > 0.0)) { why = "gamma must be > 0 when kT > 0"; return false; }
    return true;
}

lbmd_status chain_com_x(lbmd_handle *h, std::vector<double> &com) {
    std::vector<double> r(3 * (size_t)h->total_beads);
    lbmd_status s = lbmd_get_beads(h, r.data(), nullptr);
    if (s != LBMD_OK) return s;
    com.assign(h->cfg.n_real, 0.0);
    for (int q = 0; q < h->cfg.n_real; ++q) {
        const int a = h->offsets[q], b = h->offsets[q + 1];
        double acc = 0.0;
        for (int i = a; i < b; ++i) acc += r[3 * (size_t)i];
        com[q] = acc / (double)(b - a);
    }
    return LBMD_OK;
}

}  // namespace

lbmd_status lbmd_adjoint_required_bytes(const lbmd_handle *h, int32_t K, int32_t checkpoint_every, size_t *bytes) {
    if (!h || !bytes) return LBMD_ERR_INVALID_ARG;
    std::string why;
    if (!adjoint_ok(h, K, checkpoint_every, why)) return fail(const_cast<lbmd_handle *>(h), LBMD_ERR_INVALID_ARG, why);
    *bytes = adj_layout(h, K, checkpoint_every).total;
    return LBMD_OK;
}

lbmd_status lbmd_adjoint(lbmd_handle *h, int32_t K, int32_t C, void *scratch, size_t scratch_bytes, double *loss,
                         double *dgamma, double *dE, double *dr0) {
    if (!h) return LBMD_ERR_INVALID_ARG;
    if (not_slab(h, "lbmd_adjoint") != LBMD_OK) return LBMD_ERR_INVALID_ARG;
    std::string why;
    if (!adjoint_ok(h, K, C, why)) return fail(h, LBMD_ERR_INVALID_ARG, why);
    const AdjLayout a = adj_layout(h, K, C);
    if (!scratch || scratch_bytes < a.total || ((uintptr_t)scratch & 255))
        return fail(h, LBMD_ERR_BUFFER, "adjoint scratch missing, too small or not 256-byte aligned");
    char *b = (char *)scratch;
    Sim &S = h->S;
    const int n_real = h->cfg.n_real, TB = h->total_beads;
    const long long step0 = h->host_step;
    lbmd_status st = LBMD_OK;

    auto save = [&](int j) -> lbmd_status {
        char *c = b + a.ck + (size_t)j * a.ck_rec;
        char *cb = c + align256(a.pop);
        CK(cudaMemcpyAsync(c, h->popA, a.pop, cudaMemcpyDeviceToDevice, h->st));
        CK(cudaMemcpyAsync(cb, S.r_hi, (size_t)TB * 16, cudaMemcpyDeviceToDevice, h->st));
        CK(cudaMemcpyAsync(cb + (size_t)TB * 16, S.r_lo, (size_t)TB * 16, cudaMemcpyDeviceToDevice, h->st));
        CK(cudaMemcpyAsync(cb + (size_t)TB * 32, S.v, (size_t)TB * 16, cudaMemcpyDeviceToDevice, h->st));
        return LBMD_OK;
    };
    auto restore = [&](int j, long long step) -> lbmd_status {
        h->lists_ready = false;  // positions come back from a checkpoint
        const char *c = b + a.ck + (size_t)j * a.ck_rec;
        const char *cb = c + align256(a.pop);
        CK(cudaMemcpyAsync(h->popA, c, a.pop, cudaMemcpyDeviceToDevice, h->st));
        CK(cudaMemcpyAsync(S.r_hi, cb, (size_t)TB * 16, cudaMemcpyDeviceToDevice, h->st));
        CK(cudaMemcpyAsync(S.r_lo, cb + (size_t)TB * 16, (size_t)TB * 16, cudaMemcpyDeviceToDevice, h->st));
        CK(cudaMemcpyAsync(S.v, cb + (size_t)TB * 32, (size_t)TB * 16, cudaMemcpyDeviceToDevice, h->st));
        return lbmd_set_step(h, step);
    };

    // forward sweep with checkpoints
    std::vector<double> com0, comK;
    if ((st = chain_com_x(h, com0)) != LBMD_OK) return st;
    for (int n = 0; n < K; ++n) {
        if (n % C == 0 && (st = save(n / C)) != LBMD_OK) return st;
        if ((st = enqueue_step(h)) != LBMD_OK) return st;
    }
    if ((st = save(a.nck - 1)) != LBMD_OK) return st;
    if ((st = chain_com_x(h, comK)) != LBMD_OK) return st;

    // adjoint of the loss: lam_r = x^ / N_r, lam_v = 0, lam_A = 0
    float *Lin = (float *)(b + a.lamA), *Lout = (float *)(b + a.lamB);
    float4 *lam_r = (float4 *)(b + a.lam_r), *lam_v = (float4 *)(b + a.lam_v);
    unsigned long long *LU = (unsigned long long *)(b + a.LU);
    int *adj_node = (int *)(b + a.adj_node);
    double *dpar = (double *)(b + a.dpar);
    int *stamp = (int *)(b + a.stamp);
    std::vector<float4> lr0(TB);
    for (int q = 0; q < n_real; ++q)
        for (int i = h->offsets[q]; i < h->offsets[q + 1]; ++i)
            lr0[i] = make_float4((float)(1.0 / (h->offsets[q + 1] - h->offsets[q])), 0.f, 0.f, 0.f);
    CK(cudaMemsetAsync(Lin, 0, a.pop, h->st));
    CK(cudaMemsetAsync(Lout, 0, a.pop, h->st));
    CK(cudaMemsetAsync(LU, 0, (size_t)n_real * 3 * S.ns * 8, h->st));
    CK(cudaMemsetAsync(dpar, 0, (size_t)n_real * 2 * sizeof(double), h->st));
    CK(cudaMemsetAsync(stamp, 0, (size_t)n_real * S.ns * sizeof(int), h->st));
    CK(cudaMemsetAsync(lam_v, 0, (size_t)TB * 16, h->st));
    CK(cudaMemcpyAsync(lam_r, lr0.data(), (size_t)TB * 16, cudaMemcpyHostToDevice, h->st));

    // Backward sweep, segment by segment from the last.  A segment is
    // replayed from its checkpoint on the main stream, recording every
    // step's populations and the MD trajectory, then run backward on the
    // adjoint's own streams (bst, and baux for the bead adjoint beside the
    // lattice adjoint).  The replay of segment j - 1 runs while segment j
    // runs backward: the records alternate between two buffers, a replay
    // waits for the backward pass that last read its buffer, a backward pass
    // for its replay.  The backward kernels read only the records, the
    // adjoint scratch and the geometry.
    auto seg_buf = [&](int j) { return b + a.seg + (size_t)(j & 1) * a.seg_rec * a.nseg; };
    auto replay = [&](int j) -> lbmd_status {
        const int n0 = j * C, n1 = std::min(K, n0 + C);
        lbmd_status s2 = restore(j, step0 + n0);
        if (s2 != LBMD_OK) return s2;
        for (int n = n0; n < n1; ++n) {
            char *rec = seg_buf(j) + (size_t)(n - n0) * a.seg_rec;
            CK(cudaMemcpyAsync(rec, h->popA, a.pop, cudaMemcpyDeviceToDevice, h->st));
            S.traj = (float4 *)(rec + align256(a.pop));
            s2 = enqueue_step(h);
            S.traj = nullptr;
            if (s2 != LBMD_OK) return s2;
        }
        CK(cudaEventRecord(h->ev_rep[j & 1], h->st));
        return LBMD_OK;
    };
    CK(cudaEventRecord(h->ev_bstart, h->st));  // the adjoint's starting values are set
    CK(cudaStreamWaitEvent(h->bst, h->ev_bstart, 0));
    const int jl = (K - 1) / C;
    if ((st = replay(jl)) != LBMD_OK) return st;
    for (int j = jl; j >= 0; --j) {
        const int n0 = j * C, n1 = std::min(K, n0 + C);
        CK(cudaStreamWaitEvent(h->bst, h->ev_rep[j & 1], 0));
        for (int n = n1 - 1; n >= n0; --n) {
            const char *rec = seg_buf(j) + (size_t)(n - n0) * a.seg_rec;
            const void *An = rec;
            const float4 *trj = (const float4 *)(rec + align256(a.pop));
            CK(cudaEventRecord(h->ev_bfork, h->bst));
            CK(cudaStreamWaitEvent(h->baux, h->ev_bfork, 0));
            {
                ProfScope ps(h, K_BEAD_ADJOINT, h->baux);
                CK(launch_bead_adjoint(S, An, Lin, trj, lam_r, lam_v, LU, adj_node, dpar, step0 + n, h->baux));
            }
            CK(cudaEventRecord(h->ev_bjoin, h->baux));
            {
                ProfScope ps(h, K_SC_ADJOINT, h->bst);
                // the adjoint pass has the scalar kernel's block shape: the
                // step's tiles where they are the scalar kernel's, else (4, 4)
                const bool scalar = h->by > 0;
                CK(launch_sc_adjoint(S, An, Lin, Lout, scalar ? h->by : 4, scalar ? h->zc : 4, h->bst));
            }
            CK(cudaStreamWaitEvent(h->bst, h->ev_bjoin, 0));
            {
                ProfScope ps(h, K_ADJ_FIXUP, h->bst);
                CK(launch_adj_fixup(S, An, Lout, adj_node, LU, stamp, -1 - (int)((step0 + n) & 0x3fffffffll), h->bst));
            }
            std::swap(Lin, Lout);
            h->launches += 3;
        }
        CK(cudaEventRecord(h->ev_bwd[j & 1], h->bst));
        if (j > 0) {
            // segment j - 1's records go where segment j + 1's were read
            if (j + 1 <= jl) CK(cudaStreamWaitEvent(h->st, h->ev_bwd[(j + 1) & 1], 0));
            if ((st = replay(j - 1)) != LBMD_OK) return st;
        }
    }
    CK(cudaStreamWaitEvent(h->st, h->ev_bwd[0], 0));  // segment 0's backward pass ends the sweep

    // outputs, and the state after the K steps
    std::vector<float4> lr(TB);
    std::vector<double> dp(2 * (size_t)n_real);
    CK(cudaMemcpyAsync(lr.data(), lam_r, (size_t)TB * 16, cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(dp.data(), dpar, dp.size() * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    if ((st = restore(a.nck - 1, step0 + K)) != LBMD_OK) return st;
    CK(cudaStreamSynchronize(h->st));
    for (int q = 0; q < n_real; ++q) {
        if (loss) loss[q] = comK[q] - com0[q];
        if (dgamma) dgamma[q] = dp[2 * q];
        if (dE) dE[q] = dp[2 * q + 1];
        const double invN = 1.0 / (h->offsets[q + 1] - h->offsets[q]);
        for (int i = h->offsets[q]; i < h->offsets[q + 1]; ++i) {
            if (!dr0) break;
            dr0[3 * (size_t)i] = (double)lr[i].x - invN;
            dr0[3 * (size_t)i + 1] = lr[i].y;
            dr0[3 * (size_t)i + 2] = lr[i].z;
        }
    }
    return lbmd_check(h);
}

lbmd_status lbmd_set_graph(lbmd_handle *h, int32_t steps_per_graph) {
    if (!h || steps_per_graph < 0 || (steps_per_graph & 1)) return LBMD_ERR_INVALID_ARG;
    if (steps_per_graph > 0 && not_slab(h, "lbmd_set_graph") != LBMD_OK) return LBMD_ERR_INVALID_ARG;
    if (!h->st) return fail(h, LBMD_ERR_INVALID_ARG, "graph capture needs a non-default stream");
    drop_graph(h);
    h->graph_steps = steps_per_graph;
    return LBMD_OK;
}

lbmd_status lbmd_set_tiles(lbmd_handle *h, int32_t by, int32_t zc) {
    if (!h) return LBMD_ERR_INVALID_ARG;
    const int aby = by < 0 ? -by : by;
    if (by == 0) {
        if (!h->tma_ok || zc < 1 || zc > 256) return LBMD_ERR_INVALID_ARG;
    } else if (by < 0 && (!x2_lattice_ok(h->S) || by < -8)) {
        return LBMD_ERR_INVALID_ARG;
    } else if (!(aby == 1 || aby == 2 || aby == 4 || aby == 8 || aby == 16) || zc < 1 || zc > 64) {
        return LBMD_ERR_INVALID_ARG;
    }
    if (by != h->by || zc != h->zc) drop_graph(h);
    h->by = by;
    h->zc = zc;
    return LBMD_OK;
}

lbmd_status lbmd_set_md_shape(lbmd_handle *h, int32_t T, int32_t C) {
    if (!h || !(T == 0 || T == 1 || T == 2 || T == 4 || T == 8) || C < 0 || C > MAX_CLUSTER) return LBMD_ERR_INVALID_ARG;
    Sim trial = h->S;
    trial.md_T = T;
    trial.md_C = C;
    trial.md_bw = h->md_bonded;  // the caller's bonded mode, not an autotuned one
    const MdShape m = md_shape(trial);
    if (m.threads > 512 || m.C < 1 || m.C > MAX_CLUSTER || m.smem > 200 * 1024)
        return fail(h, LBMD_ERR_INVALID_ARG, "particle-kernel shape needs more than 512 threads per block");
    if (T != h->S.md_T || C != h->S.md_C || trial.md_bw != h->S.md_bw) drop_graph(h);
    h->S.md_T = T;
    h->S.md_C = C;
    h->S.md_bw = trial.md_bw;
    h->md_fixed = T != 0 || C != 0;
    return upload_md_map(h, h->S, 0);
}

lbmd_status lbmd_set_md_exchange(lbmd_handle *h, int32_t mode) {
    if (!h || mode < 0 || mode > 2) return LBMD_ERR_INVALID_ARG;
    h->md_exchange = mode;
    if (mode == 0) return LBMD_OK;
    const int pull = mode == 2 ? 1 : 0;
    if (pull != h->S.md_pull) drop_graph(h);
    h->S.md_pull = pull;
    return LBMD_OK;
}

lbmd_status lbmd_set_md_bonded(lbmd_handle *h, int32_t mode) {
    if (!h || mode < 0 || mode > 2) return LBMD_ERR_INVALID_ARG;
    Sim trial = h->S;
    trial.md_bw = mode;
    if (md_shape(trial).threads > 512)
        return fail(h, LBMD_ERR_INVALID_ARG, "particle-kernel shape needs more than 512 threads per block");
    if (mode != h->S.md_bw) drop_graph(h);
    h->S.md_bw = mode;
    h->md_bonded = mode;
    return LBMD_OK;
}

lbmd_status lbmd_get_md_bonded(lbmd_handle *h, int32_t *mode) {
    if (!h || !mode) return LBMD_ERR_INVALID_ARG;
    *mode = md_shape(h->S).bw ? 2 : 1;
    return LBMD_OK;
}

lbmd_status lbmd_set_md_reserve(lbmd_handle *h, int32_t mode) {
    if (!h || mode < 0 || mode > 2) return LBMD_ERR_INVALID_ARG;
    h->md_reserve = mode;
    if (mode == 0) return LBMD_OK;
    if ((mode == 2) != (h->S.md_reserve != 0)) drop_graph(h);
    h->S.md_reserve = mode == 2 ? 1 : 0;
    return LBMD_OK;
}

lbmd_status lbmd_set_wait_probe(lbmd_handle *h, int32_t on) {
    if (!h || on < 0 || on > 1) return LBMD_ERR_INVALID_ARG;
    if ((on != 0) != (h->S.wait_probe != 0)) drop_graph(h);
    h->S.wait_probe = on;
    return LBMD_OK;
}

lbmd_status lbmd_get_md_reserve(lbmd_handle *h, int32_t *reserve) {
    if (!h || !reserve) return LBMD_ERR_INVALID_ARG;
    *reserve = h->S.md_reserve ? 1 : 0;
    return LBMD_OK;
}

lbmd_status lbmd_get_md_exchange(lbmd_handle *h, int32_t *mode) {
    if (!h || !mode) return LBMD_ERR_INVALID_ARG;
    *mode = h->S.md_pull ? 2 : 1;
    return LBMD_OK;
}

lbmd_status lbmd_set_overlap(lbmd_handle *h, int32_t overlap) {
    if (!h || overlap < 0 || overlap > 1) return LBMD_ERR_INVALID_ARG;
    if ((overlap != 0) != h->overlap) drop_graph(h);
    h->overlap = overlap != 0;
    return LBMD_OK;
}

lbmd_status lbmd_get_overlap(lbmd_handle *h, int32_t *overlap) {
    if (!h || !overlap) return LBMD_ERR_INVALID_ARG;
    *overlap = h->overlap ? 1 : 0;
    return LBMD_OK;
}

lbmd_status lbmd_get_md_shape(lbmd_handle *h, int32_t *T, int32_t *C) {
    if (!h || !T || !C) return LBMD_ERR_INVALID_ARG;
    const MdShape m = md_shape(h->S);
    *T = m.T;
    *C = m.C;
    return LBMD_OK;
}

lbmd_status lbmd_get_tiles(lbmd_handle *h, int32_t *by, int32_t *zc) {
    if (!h || !by || !zc) return LBMD_ERR_INVALID_ARG;
    *by = h->by;
    *zc = h->zc;
    return LBMD_OK;
}

lbmd_status lbmd_autotune(lbmd_handle *h, int32_t reps, int32_t *by_out, int32_t *zc_out) {
    if (!h || reps < 1) return LBMD_ERR_INVALID_ARG;
    // The timed lattice passes add into the per-step fluid accumulators: they
    // are cleared before returning.
    auto put_back = [&]() -> cudaError_t {
        cudaError_t e = cudaMemsetAsync(h->S.fsum, 0, (size_t)h->cfg.n_real * 4 * sizeof(long long), h->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
        return e;
    };
    // no k_lists of a step may still be writing the list arrays while the
    // candidates' own builds run
    if (h->total_beads > 0 && h->lists_ready) CK(cudaStreamWaitEvent(h->st, h->ev_lists, 0));
    static const int BYS[] = {1, 2, 4, 8, 16};
    static const int ZCS[] = {1, 2, 4, 8, 16, 32};
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    float best = 1e30f;
    int bb = h->by, bz = h->zc;
    for (int by : BYS)
        for (int zc : ZCS) {
            if (zc > h->cfg.nz) continue;
            // warm-up, then time reps launches; B is scratch until the next step overwrites it
            CK(lattice_pass(h, h->S, by, zc, true));
            CK(cudaEventRecord(a, h->st));
            for (int k = 0; k < reps; ++k) CK(lattice_pass(h, h->S, by, zc, true));
            CK(cudaEventRecord(b, h->st));
            CK(cudaEventSynchronize(b));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, a, b));
            h->launches += reps + 1;
            if (ms < best) { best = ms; bb = by; bz = zc; }
        }
    // two x sites per thread (tiles (-by, zc))
    for (int by : BYS)
        for (int zc : ZCS) {
            if (!x2_lattice_ok(h->S) || by > 8 || zc > h->cfg.nz) break;
            CK(lattice_pass(h, h->S, -by, zc, true));
            CK(cudaEventRecord(a, h->st));
            for (int k = 0; k < reps; ++k) CK(lattice_pass(h, h->S, -by, zc, true));
            CK(cudaEventRecord(b, h->st));
            CK(cudaEventSynchronize(b));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, a, b));
            h->launches += reps + 1;
            if (ms < best) { best = ms; bb = -by; bz = zc; }
        }
    // the tensor-copy kernel, row groups per thread block
    static const int GROUPS[] = {2, 4, 8, 16, 32, 64};
    for (int g : GROUPS) {
        if (!h->tma_ok) break;
        CK(lattice_pass(h, h->S, 0, g, true));
        CK(cudaEventRecord(a, h->st));
        for (int k = 0; k < reps; ++k) CK(lattice_pass(h, h->S, 0, g, true));
        CK(cudaEventRecord(b, h->st));
        CK(cudaEventSynchronize(b));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, a, b));
        h->launches += reps + 1;
        if (ms < best) { best = ms; bb = 0; bz = g; }
    }
    lbmd_status s = lbmd_set_tiles(h, bb, bz);
    if (s != LBMD_OK) { cudaEventDestroy(a); cudaEventDestroy(b); return s; }
    if (by_out) *by_out = bb;
    if (zc_out) *zc_out = bz;
    if (h->total_beads == 0 || h->md_fixed) {  // no chain, or a shape the caller fixed
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        CK(put_back());
        return LBMD_OK;
    }
    // Particle-kernel shape: time pseudo-steps (gather, then the particle
    // kernel concurrent with the lattice pass and the bead diagnostics, as in
    // a step) for every admissible (lanes per bead, blocks per chain); the
    // bead state, the translocation records and the diagnostics ring slot the
    // pseudo-steps write (the current step's; once the ring has wrapped it
    // holds the oldest row a caller can still read) are saved and restored,
    // and G cleared, so the state is unchanged.
    const size_t bb16 = (size_t)h->total_beads * 16;
    const int R = h->cfg.n_real;
    std::vector<lbmd_transloc> tl_saved((size_t)R);
    CK(cudaMemcpyAsync(tl_saved.data(), h->S.tl, tl_saved.size() * sizeof(lbmd_transloc), cudaMemcpyDeviceToHost,
                       h->st));
    const size_t drow = sizeof(lbmd_diag);
    lbmd_diag *slot = h->S.ring + (size_t)(h->host_step % LBMD_DIAG_RING);
    std::vector<lbmd_diag> row_saved((size_t)R);
    CK(cudaMemcpy2DAsync(row_saved.data(), drow, slot, (size_t)LBMD_DIAG_RING * drow, drow, R, cudaMemcpyDeviceToHost,
                         h->st));
    char *snap = h->dbuf + h->L.snap;
    CK(cudaMemcpyAsync(snap, h->S.r_hi, bb16, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(snap + bb16, h->S.r_lo, bb16, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(snap + 2 * bb16, h->S.v, bb16, cudaMemcpyDeviceToDevice, h->st));
    // Time reps pseudo-steps of one candidate shape (a warm-up pass, then the
    // timed one) into ms.
    auto time_candidate = [&](Sim &trial, float &ms) -> cudaError_t {
        if (upload_md_map(h, trial, 1) != LBMD_OK) return cudaErrorUnknown;
        cudaError_t e = cudaSuccess;
        if (md_shape(trial).C > 8) {  // a non-portable cluster size: only where the device can place one
            int fit = 0;
            e = particles_clusters_fit(trial, &fit);
            if (e != cudaSuccess) return e;
            if (fit < 1) return cudaErrorInvalidConfiguration;
        }
#define CKT(call) do { e = (call); if (e != cudaSuccess) return e; } while (0)
        for (int pass = 0; pass < 2; ++pass) {
            CKT(cudaEventRecord(a, h->st));
            for (int k = 0; k < reps; ++k) {
                CKT(launch_lists(trial, h->st));
                CKT(launch_gather(trial, h->popA, h->st));
                CKT(cudaEventRecord(h->ev_fork, h->st));
                CKT(cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
                CKT(launch_particles(trial, h->popA, h->aux));
                CKT(cudaEventRecord(h->ev_join, h->aux));
                CKT(cudaStreamWaitEvent(h->aux2, h->ev_fork, 0));
                CKT(launch_bead_diag(trial, h->aux2));
                CKT(cudaEventRecord(h->ev_join2, h->aux2));
                if (!h->overlap) CKT(cudaStreamWaitEvent(h->st, h->ev_join, 0));
                CKT(lattice_pass(h, trial, h->by, h->zc, false));
                CKT(cudaStreamWaitEvent(h->st, h->ev_join, 0));
                CKT(cudaStreamWaitEvent(h->st, h->ev_join2, 0));
            }
            CKT(cudaEventRecord(b, h->st));
            CKT(cudaEventSynchronize(b));
            CKT(cudaEventElapsedTime(&ms, a, b));
            h->launches += 5LL * reps;
        }
#undef CKT
        return cudaSuccess;
    };
    static const int TS[] = {1, 2, 4, 8};
    static const int CS[] = {1, 2, 4, 8, 16};
    float best_md = 1e30f;
    int bt = 0, bc = 0, bx = h->S.md_pull, bb_w = h->S.md_bw, brs = h->S.md_reserve;
    for (int T : TS)
        for (int C : CS)
          for (int R = 0; R < 2; ++R)
          for (int B = 1; B <= 2; ++B)
          for (int X = 0; X < 2; ++X) {
            // both bonded modes and both SM uses unless the caller fixed one
            if (h->md_bonded != 0 && B != h->md_bonded) continue;
            if (h->md_reserve != 0 && R != h->md_reserve - 1) continue;
            // both exchanges for a chain over several blocks, unless the
            // caller fixed one; a single block exchanges nothing
            const int pull = h->md_exchange == 0 ? X : (h->md_exchange == 2 ? 1 : 0);
            if (X == 1 && (h->md_exchange != 0 || C == 1)) continue;
            Sim trial = h->S;
            trial.md_T = T;
            trial.md_C = C;
            trial.md_pull = pull;
            trial.md_bw = B;
            trial.md_reserve = R;
            const MdShape m = md_shape(trial);
            if (m.threads > 512 || m.C != C || m.smem > 200 * 1024) continue;
            if (C > 1 && C > (h->S.max_beads + 15) / 16) continue;  // blocks of a few beads: barrier-bound
            // a candidate the device cannot set up or launch is skipped; the
            // bead state is restored below whatever happened here
            float ms = 0.f;
            if (time_candidate(trial, ms) != cudaSuccess) {
                cudaGetLastError();  // clear a launch-configuration error
                continue;
            }
            // reserving SMs takes them from the lattice pass: it must win by 1%
            if (R) ms *= 1.01f;
            if (ms < best_md) { best_md = ms; bt = T; bc = C; bx = pull; bb_w = B; brs = R; }
          }
    CK(cudaMemcpyAsync(h->S.r_hi, snap, bb16, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(h->S.r_lo, snap + bb16, bb16, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(h->S.v, snap + 2 * bb16, bb16, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemsetAsync(h->S.G, 0, (size_t)h->cfg.n_real * 3 * h->S.ns * 8, h->st));
    CK(cudaMemcpyAsync(h->S.tl, tl_saved.data(), tl_saved.size() * sizeof(lbmd_transloc), cudaMemcpyHostToDevice,
                       h->st));
    CK(cudaMemcpy2DAsync(slot, (size_t)LBMD_DIAG_RING * drow, row_saved.data(), drow, drow, R, cudaMemcpyHostToDevice,
                         h->st));
    CK(put_back());
    h->lists_ready = false;  // the candidates' lists are of their pseudo-steps' positions
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (bt > 0 &&
        (bt != h->S.md_T || bc != h->S.md_C || bx != h->S.md_pull || bb_w != h->S.md_bw || brs != h->S.md_reserve)) {
        h->S.md_T = bt;
        h->S.md_C = bc;
        h->S.md_pull = bx;
        h->S.md_bw = bb_w;
        h->S.md_reserve = brs;
        drop_graph(h);
        return upload_md_map(h, h->S, 0);
    }
    return LBMD_OK;
}

lbmd_status lbmd_profile(lbmd_handle *h, int32_t enable) {
    if (!h) return LBMD_ERR_INVALID_ARG;
    lbmd_status s = resolve_profile(h);
    if (s != LBMD_OK) return s;
    if (enable && !h->profiling) {
        for (int k = 0; k < K_COUNT; ++k) { h->prof_ms[k] = 0; h->prof_n[k] = 0; }
        CK(cudaMemsetAsync(h->dbuf + h->L.phase, 0, PHASES * sizeof(unsigned long long), h->st));
    }
    h->profiling = enable != 0;
    h->S.phase = h->profiling ? (unsigned long long *)(h->dbuf + h->L.phase) : nullptr;
    drop_graph(h);
    return LBMD_OK;
}

lbmd_status lbmd_kernel_times(lbmd_handle *h, lbmd_kernel_time *out, int32_t max_entries, int32_t *n_entries) {
    if (!h || !n_entries || (max_entries > 0 && !out)) return LBMD_ERR_INVALID_ARG;
    lbmd_status s = resolve_profile(h);
    if (s != LBMD_OK) return s;
    static const char *PNAMES[PHASES - 1] = {"particles.load", "particles.lists", "particles.md", "particles.spread",
                                             "particles.rebuilds"};
    unsigned long long cyc[PHASES] = {0, 0, 0, 0, 0, 0};
    CK(cudaMemcpyAsync(cyc, h->dbuf + h->L.phase, sizeof(cyc), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    int dev = 0, khz = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
    int n = 0;
    auto put = [&](const char *name, long long launches, double ms) {
        if (n >= max_entries) return;
        memset(out[n].name, 0, sizeof(out[n].name));
        strncpy(out[n].name, name, sizeof(out[n].name) - 1);
        out[n].launches = launches;
        out[n].total_ms = ms;
        ++n;
    };
    for (int k = 0; k < K_COUNT; ++k) put(KNAMES[k], h->prof_n[k], h->prof_ms[k]);
    // phases 0..4 are SM cycles; slot 5 counts the list rebuilds (reported as
    // the "launches" of particles.rebuilds)
    for (int k = 0; k < PHASES - 1; ++k)
        put(PNAMES[k], k == 4 ? (long long)cyc[5] : h->prof_n[K_PARTICLES],
            khz > 0 ? (double)cyc[k] / (double)khz : 0.0);
    *n_entries = n;
    return LBMD_OK;
}

lbmd_status lbmd_launch_count(lbmd_handle *h, int64_t *launches) {
    if (!h || !launches) return LBMD_ERR_INVALID_ARG;
    *launches = h->launches;
    return LBMD_OK;
}

lbmd_status lbmd_slab_buffers(lbmd_handle *h, lbmd_slab_io *io) {
    if (slab_only(h) != LBMD_OK || !io) return LBMD_ERR_INVALID_ARG;
    io->up = reinterpret_cast<float *>(h->S.up);
    io->send_lo = h->dbuf + h->L.xsend_lo;
    io->send_hi = h->dbuf + h->L.xsend_hi;
    io->recv_lo = h->dbuf + h->L.xrecv_lo;
    io->recv_hi = h->dbuf + h->L.xrecv_hi;
    io->plane_bytes = (size_t)LBMD_Q * h->S.ny * h->S.nz * (h->cfg.precision == LBMD_FP16DEV ? 2 : 4);
    return LBMD_OK;
}

lbmd_status lbmd_slab_gather(lbmd_handle *h) {
    if (slab_only(h) != LBMD_OK) return LBMD_ERR_INVALID_ARG;
    return enqueue_gather(h);
}

lbmd_status lbmd_slab_advance(lbmd_handle *h) {
    if (slab_only(h) != LBMD_OK) return LBMD_ERR_INVALID_ARG;
    lbmd_status s = enqueue_advance(h);
    if (s != LBMD_OK) return s;
    // the step's result (now in A): local planes 1, 2 for the left
    // neighbour, the last own plane for the right one
    const int w = h->cfg.slab_nx;
    CK(launch_slab_planes(h->S, h->popA, h->dbuf + h->L.xsend_lo, 1, 2, true, h->st));
    CK(launch_slab_planes(h->S, h->popA, h->dbuf + h->L.xsend_hi, w, 1, true, h->st));
    h->launches += 2;
    return LBMD_OK;
}

lbmd_status lbmd_slab_import(lbmd_handle *h) {
    if (slab_only(h) != LBMD_OK) return LBMD_ERR_INVALID_ARG;
    const int w = h->cfg.slab_nx;
    CK(launch_slab_planes(h->S, h->popA, h->dbuf + h->L.xrecv_lo, 0, 1, false, h->st));
    CK(launch_slab_planes(h->S, h->popA, h->dbuf + h->L.xrecv_hi, w + 1, 2, false, h->st));
    h->launches += 2;
    return LBMD_OK;
}

void lbmd_destroy(lbmd_handle *h) {
    if (!h) return;
    if (h->st) cudaStreamSynchronize(h->st);
    if (h->aux) cudaStreamSynchronize(h->aux);
    if (h->aux2) cudaStreamSynchronize(h->aux2);
    if (h->bst) cudaStreamSynchronize(h->bst);
    if (h->baux) cudaStreamSynchronize(h->baux);
    for (auto &p : h->pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : h->free_events) cudaEventDestroy(e);
    drop_graph(h);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->ev_join2) cudaEventDestroy(h->ev_join2);
    if (h->ev_pre) cudaEventDestroy(h->ev_pre);
    if (h->ev_lists) cudaEventDestroy(h->ev_lists);
    if (h->ev_lists_cap) cudaEventDestroy(h->ev_lists_cap);
    for (cudaEvent_t ev : {h->ev_bfork, h->ev_bjoin, h->ev_bstart, h->ev_rep[0], h->ev_rep[1], h->ev_bwd[0], h->ev_bwd[1]})
        if (ev) cudaEventDestroy(ev);
    if (h->aux) cudaStreamDestroy(h->aux);
    if (h->aux2) cudaStreamDestroy(h->aux2);
    if (h->bst) cudaStreamDestroy(h->bst);
    if (h->baux) cudaStreamDestroy(h->baux);
    delete h;
}

}  // extern "C"
