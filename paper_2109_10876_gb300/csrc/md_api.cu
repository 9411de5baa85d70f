// Host side of the C ABI declared in include/md.h: parameter checks, the
// cell grid of every replica (edge >= r_cut + r_skin, Sec. 2.1.2 of
// arXiv:2109.10876), device allocations owned by the handle, and the kernel
// sequence of one velocity-Verlet step (Fig. 1).
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "md.h"
#include "md_internal.cuh"

using mdk::Bufs;
using mdk::Ctl;
using mdk::Replica;

struct md_handle {
    md_params p{};
    std::vector<Replica> reps;
    std::vector<int64_t> offsets;
    Bufs b{};
    std::vector<void *> allocs;
    int precision = 1;
    bool auto_capacity = true;
    bool state_set = false;
    bool F_valid = false;
    bool built = false;   // a growing list build (md_build_neighbors) ran since the last md_set_state
    long long N = 0, S = 0;
    int C = 0, nblk = 0, K = 0, nrows = 0;
    double *stage = nullptr;        // 6 * N doubles: in/out staging
    double *thermo_stage = nullptr; // grows on demand
    long long thermo_cap = 0;
    unsigned long long *d_count = nullptr;
    std::string err;
    // section timers: event pairs recorded in md_step, resolved in md_get_timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<std::pair<int, std::pair<size_t, size_t>>> ev_marks;   // (section, (start, stop))
    double sect_ms[MD_NSECT] = {0, 0, 0};
    long long sect_n[MD_NSECT] = {0, 0, 0};
    // recorded differentiable run (md_forward) for md_backward
    bool ad_ready = false;
    int ad_T = 0, ad_k = 1;
    double *ad_ck = nullptr;        // checkpoints: (x, v) in caller order, 6 N each
    long long ad_ck_cap = 0;        // checkpoints the buffer holds
    double *ad_fin = nullptr;       // final (x, v), 6 N
    double *ad_work = nullptr;      // lx, lv, hv: 3 x 3 N
    double *ad_seg = nullptr;       // positions of one segment: (k + 1) x 3 N
    long long ad_seg_cap = 0;
    double *ad_small = nullptr;     // coef (4 nrep), g (4 nrep), sums (4 nrep)
    // the step loop as a CUDA graph (conditional WHILE over steps, IF over rebuilds)
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr, gexec_e = nullptr;       // without / with energies every step
    cudaGraph_t graph_e = nullptr;
    long long gen = 0, gexec_gen = -1, gexec_e_gen = -1;   // gen: bumped whenever the kernels' buffers change
    // the step graph that also records the positions after every step (the
    // reverse pass's segment re-runs, into ad_seg)
    cudaGraph_t graph_x = nullptr;
    cudaGraphExec_t gexec_x = nullptr;
    long long gexec_x_gen = -1;
    // the rebuild chain alone behind a conditional IF (the reverse pass's reloads)
    cudaGraph_t graph_chain = nullptr;
    cudaGraphExec_t gexec_chain = nullptr;
    long long gexec_chain_gen = -1;
    bool use_graph = true;
    // md_set_recovery: md_step grows the list / halo capacity and finishes the
    // call when a rebuild inside it overflowed
    bool recover = false;
    long long recoveries = 0;
};

namespace {

md_status fail(md_handle *h, md_status s, const std::string &msg)
{
    if (h) h->err = msg;
    return s;
}

bool cuda_ok(md_handle *h, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return true;
    if (h) h->err = std::string(what) + ": " + cudaGetErrorString(e);
    return false;
}

template <class T>
T *dalloc(md_handle *h, size_t count)
{
    void *p = nullptr;
    if (count == 0) count = 1;
    if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) return nullptr;
    h->allocs.push_back(p);
    return static_cast<T *>(p);
}

double lj_v(double r, double eps, double sig)
{
    double s6 = std::pow(sig / r, 6.0);
    return 4.0 * eps * (s6 * s6 - s6);
}

double lj_fmag(double r, double eps, double sig)
{
    double s6 = std::pow(sig / r, 6.0);
    return 24.0 * eps * (2.0 * s6 * s6 - s6) / r;
}

long long round_up(long long a, long long m) { return (a + m - 1) / m * m; }

static_assert(mdk::kSiteBinCell == MD_SITE_BIN_CELL && mdk::kSiteScatter == MD_SITE_SCATTER &&
                  mdk::kSiteReorder == MD_SITE_REORDER && mdk::kSiteTopology == MD_SITE_TOPOLOGY &&
                  mdk::kSiteTileWrite == MD_SITE_TILE_WRITE && mdk::kSitePieces == MD_SITE_PIECES &&
                  mdk::kSiteListRange == MD_SITE_LIST_RANGE && mdk::kSiteListSelf == MD_SITE_LIST_SELF &&
                  mdk::kSiteForceHalo == MD_SITE_FORCE_HALO && mdk::kSiteForceOwn == MD_SITE_FORCE_OWN &&
                  mdk::kSiteForceSlot == MD_SITE_FORCE_SLOT && mdk::kSiteBondSlot == MD_SITE_BOND_SLOT &&
                  mdk::kSiteAdjHalo == MD_SITE_ADJ && mdk::kSiteCount == MD_SITE_ADJ + 1,
              "check sites of md.h and of the kernels agree");

const char *site_name(int site)
{
    static const char *names[mdk::kSiteCount] = {
        "none",
        "cell of a particle (binning)",
        "bucket slot (scatter)",
        "particle id or destination slot (re-sort)",
        "bond or angle partner id (topology)",
        "tile index (tiling)",
        "halo piece (tiling)",
        "candidate range in the halo (list build)",
        "own halo entries (list build)",
        "list entry in the halo (force)",
        "own halo entry (force)",
        "slot of a halo entry (force)",
        "bond or angle partner slot (force)",
        "list entry, id or slot (reverse pass)",
    };
    return site > 0 && site < mdk::kSiteCount ? names[site] : "unknown";
}

// Map latched device error bits to a status.
md_status status_of(md_handle *h, const Ctl &c)
{
    const int bits = c.err;
    if (!bits) return MD_OK;
    if (bits & mdk::kErrBounds) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "device bounds check failed: site %d (%s), index %lld", c.bad_site,
                      site_name(c.bad_site), (long long)c.bad_index);
        return fail(h, MD_ERR_BOUNDS, msg);
    }
    if (bits & mdk::kErrList) return fail(h, MD_ERR_LIST_OVERFLOW, "neighbour list capacity exceeded");
    if (bits & mdk::kErrBond) return fail(h, MD_ERR_BOND_BROKEN, "FENE bond reached r >= R0");
    if (bits & mdk::kErrFixed) return fail(h, MD_ERR_FIXED_OVERFLOW, "pair force outside the fixed-point range");
    if (bits & mdk::kErrNonfinite) return fail(h, MD_ERR_NONFINITE, "non-finite position, velocity or force");
    if (bits & mdk::kErrTimeout) return fail(h, MD_ERR_TIMEOUT, "bounded device wait timed out");
    return fail(h, MD_ERR_CUDA, "unknown device error bits");
}

md_status read_ctl(md_handle *h, Ctl *out)
{
    if (!cuda_ok(h, cudaMemcpy(out, h->b.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost), "read control block"))
        return MD_ERR_CUDA;
    return MD_OK;
}

md_status alloc_list(md_handle *h, int K)
{
    if (h->b.nbr) {
        for (auto it = h->allocs.begin(); it != h->allocs.end(); ++it)
            if (*it == h->b.nbr) { cudaFree(*it); h->allocs.erase(it); break; }
        h->b.nbr = nullptr;
    }
    h->K = K;
    h->b.K = K;
    h->gen++;
    // 16 entries of slack: the force kernel's bulk copy of a tile's list block
    // rounds its length up to 16 bytes
    h->b.nbr = dalloc<unsigned short>(h, (size_t)K * (size_t)h->S + 16);
    if (!h->b.nbr) return fail(h, MD_ERR_CUDA, "cannot allocate the neighbour list");
    return MD_OK;
}

md_status ensure_thermo(md_handle *h, long long count)
{
    if (h->thermo_cap >= count) return MD_OK;
    if (h->thermo_stage) {
        for (auto it = h->allocs.begin(); it != h->allocs.end(); ++it)
            if (*it == h->thermo_stage) { cudaFree(*it); h->allocs.erase(it); break; }
        h->thermo_stage = nullptr;
        h->thermo_cap = 0;
    }
    h->thermo_stage = dalloc<double>(h, (size_t)count);
    if (!h->thermo_stage) return fail(h, MD_ERR_CUDA, "cannot allocate thermo buffer");
    h->thermo_cap = count;
    h->gen++;   // the energy graph holds the buffer's address
    return MD_OK;
}

double *grow(md_handle *h, double *old, size_t count)
{
    if (old) {
        for (auto it = h->allocs.begin(); it != h->allocs.end(); ++it)
            if (*it == old) { cudaFree(*it); h->allocs.erase(it); break; }
    }
    return dalloc<double>(h, count);
}

cudaEvent_t next_event(md_handle *h)
{
    if (h->ev_used == h->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        h->ev_pool.push_back(e);
    }
    return h->ev_pool[h->ev_used++];
}

// record a timing mark on the stream; returns its pool index (or -1)
long long mark(md_handle *h, cudaStream_t st)
{
    if (!h->timing) return -1;
    cudaEvent_t e = next_event(h);
    if (!e) return -1;
    cudaEventRecord(e, st);
    return (long long)h->ev_used - 1;
}

void section(md_handle *h, int sect, long long a, long long b)
{
    if (a >= 0 && b >= 0) h->ev_marks.push_back({sect, {(size_t)a, (size_t)b}});
}

// fold recorded marks into the accumulated section times (events complete)
void resolve_timing(md_handle *h)
{
    for (auto &m : h->ev_marks) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev_pool[m.second.first], h->ev_pool[m.second.second]) == cudaSuccess) {
            h->sect_ms[m.first] += ms;
            h->sect_n[m.first] += 1;
        }
    }
    h->ev_marks.clear();
    h->ev_used = 0;
}

md_status sync_and_check(md_handle *h, cudaStream_t st)
{
    if (!cuda_ok(h, cudaStreamSynchronize(st), "stream synchronize")) return MD_ERR_CUDA;
    if (!cuda_ok(h, cudaGetLastError(), "kernel launch")) return MD_ERR_CUDA;
    Ctl c;
    md_status s = read_ctl(h, &c);
    if (s != MD_OK) return s;
    return status_of(h, c);
}

// Capture f(stream) into graph g after deps; tail gets the captured sink nodes.
template <class F>
bool capture_into(md_handle *h, cudaGraph_t g, const std::vector<cudaGraphNode_t> &deps, F f,
                  std::vector<cudaGraphNode_t> *tail)
{
    if (cudaStreamBeginCaptureToGraph(h->cap, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                                      cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return false;
    f(h->cap);
    if (tail) {
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t *d = nullptr;
        size_t nd = 0;
        if (cudaStreamGetCaptureInfo(h->cap, &cs, nullptr, nullptr, &d, nullptr, &nd) != cudaSuccess) return false;
        tail->assign(d, d + nd);
    }
    cudaGraph_t out = nullptr;
    return cudaStreamEndCapture(h->cap, &out) == cudaSuccess;
}

// One graph for md_step(n > 0) without timers, without energies or with
// energies every step (`energy`):
//   kick-drift -> cond(W: steps left) -> WHILE(W) { cond(I: rebuild) -> IF(I) { rebuild chain }
//   -> fused force } -> cond(I2) -> IF(I2) { rebuild chain } -> final force.
// The fused kernel's last block counts the steps down and sets W; with
// energies, each force kernel's last block writes its record to the next slot
// of the thermo buffer.  With `record` (no energies), the positions after the
// kick-drift and after every fused force are written to the slots of the
// reverse pass's segment buffer (k_record_x, slot = steps since the call began).
bool build_step_graph(md_handle *h, bool energy, bool record = false)
{
    cudaGraphExec_t &gexec = record ? h->gexec_x : energy ? h->gexec_e : h->gexec;
    cudaGraph_t &graph = record ? h->graph_x : energy ? h->graph_e : h->graph;
    long long &ggen = record ? h->gexec_x_gen : energy ? h->gexec_e_gen : h->gexec_gen;
    if (gexec && ggen == h->gen) return true;
    if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
    if (graph) { cudaGraphDestroy(graph); graph = nullptr; }
    if (!h->cap && cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) return false;
    cudaGraph_t G;
    if (cudaGraphCreate(&G, 0) != cudaSuccess) return false;
    graph = G;
    cudaGraphConditionalHandle hW, hI2;
    if (cudaGraphConditionalHandleCreate(&hW, G, 0, 0) != cudaSuccess) return false;
    if (cudaGraphConditionalHandleCreate(&hI2, G, 0, 0) != cudaSuccess) return false;
    Bufs b = h->b;
    b.g_while = 0;
    b.thermo = nullptr;
    b.thermo_ring = energy ? h->thermo_stage : nullptr;
    b.xring = record ? h->ad_seg : nullptr;
    const int prec = h->precision;
    std::vector<cudaGraphNode_t> tail;
    if (!capture_into(h, G, {}, [&](cudaStream_t s) {
            mdk::launch_kick_drift(b, s);
            if (record) mdk::launch_record_x(b, s);
            mdk::launch_cond(b, hW, 1, s);
        }, &tail))
        return false;
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = hW;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t nW;
    if (cudaGraphAddNode(&nW, G, tail.data(), nullptr, tail.size(), &wp) != cudaSuccess) return false;
    cudaGraph_t BW = wp.conditional.phGraph_out[0];
    cudaGraphConditionalHandle hI;
    if (cudaGraphConditionalHandleCreate(&hI, BW, 0, 0) != cudaSuccess) return false;
    if (!capture_into(h, BW, {}, [&](cudaStream_t s) { mdk::launch_cond(b, hI, 0, s); }, &tail)) return false;
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = hI;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t nI;
    if (cudaGraphAddNode(&nI, BW, tail.data(), nullptr, tail.size(), &ip) != cudaSuccess) return false;
    if (!capture_into(h, ip.conditional.phGraph_out[0], {}, [&](cudaStream_t s) { mdk::launch_rebuild_chain(b, s); },
                      nullptr))
        return false;
    Bufs bf = b;
    bf.g_while = hW;
    if (!capture_into(h, BW, {nI}, [&](cudaStream_t s) {
            mdk::launch_force(bf, prec, mdk::kModeFused, energy, s);
            if (record) mdk::launch_record_x(b, s);
        }, nullptr))
        return false;
    if (!capture_into(h, G, {nW}, [&](cudaStream_t s) { mdk::launch_cond(b, hI2, 0, s); }, &tail)) return false;
    cudaGraphNodeParams ip2 = {};
    ip2.type = cudaGraphNodeTypeConditional;
    ip2.conditional.handle = hI2;
    ip2.conditional.type = cudaGraphCondTypeIf;
    ip2.conditional.size = 1;
    cudaGraphNode_t nI2;
    if (cudaGraphAddNode(&nI2, G, tail.data(), nullptr, tail.size(), &ip2) != cudaSuccess) return false;
    if (!capture_into(h, ip2.conditional.phGraph_out[0], {}, [&](cudaStream_t s) { mdk::launch_rebuild_chain(b, s); },
                      nullptr))
        return false;
    if (!capture_into(h, G, {nI2}, [&](cudaStream_t s) { mdk::launch_force(b, prec, mdk::kModeFinal, energy, s); },
                      nullptr))
        return false;
    if (cudaGraphInstantiate(&gexec, G, 0) != cudaSuccess) { gexec = nullptr; return false; }
    ggen = h->gen;
    return true;
}

// The rebuild chain behind a conditional IF set from Ctl::rebuild, as one
// graph: where the decision to rebuild is taken on the device and most calls
// need no rebuild, one graph launch replaces the chain's kernels, each of
// which would otherwise be launched only to return at once.
bool build_chain_graph(md_handle *h)
{
    if (h->gexec_chain && h->gexec_chain_gen == h->gen) return true;
    if (h->gexec_chain) { cudaGraphExecDestroy(h->gexec_chain); h->gexec_chain = nullptr; }
    if (h->graph_chain) { cudaGraphDestroy(h->graph_chain); h->graph_chain = nullptr; }
    if (!h->cap && cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) return false;
    cudaGraph_t G;
    if (cudaGraphCreate(&G, 0) != cudaSuccess) return false;
    h->graph_chain = G;
    cudaGraphConditionalHandle hI;
    if (cudaGraphConditionalHandleCreate(&hI, G, 0, 0) != cudaSuccess) return false;
    Bufs b = h->b;
    b.g_while = 0;
    b.thermo = nullptr;
    b.thermo_ring = nullptr;
    std::vector<cudaGraphNode_t> tail;
    if (!capture_into(h, G, {}, [&](cudaStream_t s) { mdk::launch_cond(b, hI, 0, s); }, &tail)) return false;
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = hI;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t nI;
    if (cudaGraphAddNode(&nI, G, tail.data(), nullptr, tail.size(), &ip) != cudaSuccess) return false;
    if (!capture_into(h, ip.conditional.phGraph_out[0], {}, [&](cudaStream_t s) { mdk::launch_rebuild_chain(b, s); },
                      nullptr))
        return false;
    if (cudaGraphInstantiate(&h->gexec_chain, G, 0) != cudaSuccess) { h->gexec_chain = nullptr; return false; }
    h->gexec_chain_gen = h->gen;
    return true;
}

// After a list or halo overflow (c.err == kErrList): grow the list capacity
// and / or the halo capacity to fit what the failed build needed, then clear
// the error word and the sums a cut-short launch may have left behind.
md_status grow_after_overflow(md_handle *h, const Ctl &c)
{
    bool grew = false;
    if (c.max_nn > h->K) {
        int K = (int)round_up((long long)(c.max_nn * 1.25) + 32, 32);
        if (K > 65535 || alloc_list(h, K) != MD_OK) return fail(h, MD_ERR_LIST_OVERFLOW, "neighbour list too long");
        grew = true;
    }
    if (c.max_halo > h->b.hcap) {
        const int lim = (h->precision == MD_FP32_FIXED) ? 12288 : 8192;   // shared memory per block
        int hc = (int)round_up((long long)(c.max_halo * 1.25), 128);
        if (c.max_halo > lim) return fail(h, MD_ERR_LIST_OVERFLOW, "a cell neighbourhood exceeds the halo capacity");
        h->b.hcap = std::min(hc, lim);
        h->gen++;
        grew = true;
    }
    if (!grew) return fail(h, MD_ERR_LIST_OVERFLOW, "neighbour list overflow that no capacity growth covers");
    int zero = 0;
    if (!cuda_ok(h, cudaMemcpy(&h->b.ctl->err, &zero, sizeof(int), cudaMemcpyHostToDevice), "clear error"))
        return MD_ERR_CUDA;
    if (h->b.Fq && !cuda_ok(h, cudaMemset(h->b.Fq, 0, sizeof(long long) * 3 * h->S), "clear force sums"))
        return MD_ERR_CUDA;
    if (!cuda_ok(h, cudaMemset(h->b.eacc, 0, sizeof(long long) * 4 * (size_t)h->b.nrep), "clear energy sums"))
        return MD_ERR_CUDA;
    return MD_OK;
}

}  // namespace

extern "C" {

md_status md_create(const md_params *p, md_handle **out)
{
    if (!out) return MD_ERR_ARG;
    *out = nullptr;
    if (!p || p->n_replicas < 1 || p->n_replicas > mdk::kMaxReplicas || !p->replica_offsets || !p->box ||
        !p->eps || !p->sigma)
        return MD_ERR_ARG;
    if (!(p->dt > 0) || !(p->mass > 0) || !(p->skin >= 0) ||
        (p->potential != MD_LJ && p->potential != MD_WCA && p->potential != MD_SOFT) ||
        (p->precision != MD_FP64 && p->precision != MD_FP32_FIXED) || p->langevin_gamma < 0 ||
        (p->potential != MD_WCA && !(p->rc_over_sigma > 0)) ||
        (p->potential == MD_SOFT && p->precision != MD_FP64) || p->list_capacity < 0 || p->n_bonds < 0 ||
        (p->n_bonds > 0 && (!p->bonds || !(p->fene_K > 0) || !(p->fene_R0 > 0))) ||
        (p->langevin_gamma > 0 && !(p->kT >= 0)))
        return MD_ERR_ARG;
    if (p->replica_offsets[0] != 0) return MD_ERR_ARG;
    md_handle *h = new md_handle();
    h->p = *p;
    h->precision = p->precision;
    const int nrep = p->n_replicas;
    h->offsets.assign(p->replica_offsets, p->replica_offsets + nrep + 1);
    long long slot = 0;
    int cell = 0, rows = 0;
    for (int r = 0; r < nrep; ++r) {
        long long n = h->offsets[r + 1] - h->offsets[r];
        if (n < 0 || n > (1LL << 30)) { delete h; return MD_ERR_ARG; }
        Replica R{};
        const double eps = p->eps[r], sig = p->sigma[r];
        if (!(eps > 0) || !(sig > 0)) { delete h; return MD_ERR_ARG; }
        const double rc = (p->potential == MD_WCA ? std::pow(2.0, 1.0 / 6.0) : p->rc_over_sigma) * sig;
        const double rl = rc + p->skin;
        double Lmax = 0;
        for (int k = 0; k < 3; ++k) {
            const double L = p->box[3 * r + k];
            if (!(L > 0) || !std::isfinite(L)) { delete h; return MD_ERR_ARG; }
            if (L < 2.0 * rl) {
                delete h;
                return MD_ERR_BOX_TOO_SMALL;
            }
            Lmax = std::fmax(Lmax, L);
            R.L[k] = L;
            R.to_q[k] = 4294967296.0 / L;
            R.from_q[k] = L / 4294967296.0;
            R.qs[k] = (float)(L / 4294967296.0);
            // cell edge L / n >= r_cut + r_skin, with a margin far above the
            // fixed-point quantisation so that the 27-cell search is complete
            int nc = (int)std::floor(L / (rl * (1.0 + 1e-6) + 4.0 * L / 4294967296.0));
            R.ncell[k] = nc < 1 ? 1 : nc;
        }
        if ((long long)R.ncell[0] * R.ncell[1] * R.ncell[2] > (1LL << 28)) { delete h; return MD_ERR_ARG; }
        R.cell_off = cell;
        R.ncells = R.ncell[0] * R.ncell[1] * R.ncell[2];
        cell += R.ncells;
        R.row_off = rows;
        rows += R.ncell[1] * R.ncell[2];
        R.slot_begin = slot;
        R.n = n;
        R.id_begin = h->offsets[r];
        R.blk_begin = (int)(slot / mdk::kBlock);
        slot += round_up(n, mdk::kBlock);
        R.blk_end = (int)(slot / mdk::kBlock);
        R.eps = eps;
        R.sigma = sig;
        R.rc = rc;
        R.rc2 = rc * rc;
        R.soft = p->potential == MD_SOFT ? 1 : 0;
        R.vshift = R.soft ? 0.0 : lj_v(rc, eps, sig);
        R.rl2 = rl * rl;
        R.eps24_f = (float)(24.0 * eps);
        R.eps4_f = (float)(4.0 * eps);
        R.sig2_f = (float)(sig * sig);
        R.rc2_f = (float)(rc * rc);
        R.vshift_f = (float)R.vshift;
        // bands around the cutoffs inside which the FP32 r^2 cannot decide:
        // fixed-point quantisation (|dd| <= sqrt(3) L / 2^32) plus FP32 rounding
        const double qd = std::sqrt(3.0) * Lmax / 4294967296.0;
        // FP32 r^2 from exact integer differences: one rounding per component
        // and three in the sum of squares, below 5 x 2^-24 relative; 2^-20
        // leaves a factor of three
        const double brc = 2.0 * rc * qd + std::ldexp(1.0, -20) * rc * rc;
        // the list walk rounds coordinates relative to the tile centre (|c| <= L / 2)
        // to FP32: up to L / 2^24 more per separation component
        const double brl = 2.0 * rl * (qd + std::sqrt(3.0) * Lmax / 16777216.0) + std::ldexp(1.0, -20) * rl * rl;
        R.rc2_lo = (float)(rc * rc - brc);
        R.rc2_hi = (float)(rc * rc + brc);
        R.rl2_lo = (float)(rl * rl - brl);
        R.rl2_hi = (float)(rl * rl + brl);
        double half = 0.5 * p->skin * (1.0 - 1e-6) - 2.0 * qd;
        R.disp2_thr = (float)std::fmax(half * half, 1e-30);
        // smallest r^2 at which one pair-force component stays below 2^21
        double lo = 1e-3 * sig, hi = rc;
        for (int it = 0; it < 200; ++it) {
            double mid = 0.5 * (lo + hi);
            if (lj_fmag(mid, eps, sig) > std::ldexp(1.0, 21) * 0.9) lo = mid; else hi = mid;
        }
        R.fmax2 = (float)(hi * hi);
        const double u = R.L[0] / 4294967296.0;   // fixed-point unit of the x axis
        R.cubic = (R.L[0] == R.L[1] && R.L[0] == R.L[2]) ? 1 : 0;
        R.ry = (float)(R.L[1] / R.L[0]);
        R.rz = (float)(R.L[2] / R.L[0]);
        R.rc2_lo_u = (float)((rc * rc - brc) / (u * u));
        R.rc2_hi_u = (float)((rc * rc + brc) / (u * u));
        R.fmax2_u = (float)(hi * hi / (u * u));
        R.sig2_u = (float)(sig * sig / (u * u));
        R.eps24_u = (float)(24.0 * eps / u);
        R.rl2_lo_u = (float)((rl * rl - brl) / (u * u));
        R.rl2_hi_u = (float)((rl * rl + brl) / (u * u));
        // beyond this x distance no pair reaches r_list + its band, with room
        // for the FP32 rounding of tile-relative coordinates (<= 2^8 u per entry)
        R.rl_win_u = (float)(rl * (1.0 + std::ldexp(1.0, -14)) / u + 2048.0);
        h->reps.push_back(R);
    }
    h->N = h->offsets[nrep];
    h->S = slot;
    h->C = cell;
    h->nrows = rows;
    h->nblk = (int)(slot / mdk::kBlock);
    if (h->N < 1) { delete h; return MD_ERR_ARG; }

    // FENE bonds must join two distinct particles of the same replica
    for (int64_t q = 0; q < p->n_bonds; ++q) {
        long long a = p->bonds[2 * q], c = p->bonds[2 * q + 1];
        if (a < 0 || c < 0 || a >= h->N || c >= h->N || a == c) { delete h; return MD_ERR_ARG; }
        int ra = 0, rb = 0;
        while (h->offsets[ra + 1] <= a) ++ra;
        while (h->offsets[rb + 1] <= c) ++rb;
        if (ra != rb) { delete h; return MD_ERR_ARG; }
    }

    // angle triples: three distinct particles of one replica
    if (p->n_angles < 0 || (p->n_angles > 0 && !p->angles) || (p->n_angles > 0 && !(p->angle_K >= 0))) {
        delete h;
        return MD_ERR_ARG;
    }
    for (int64_t q = 0; q < p->n_angles; ++q) {
        long long id3[3];
        int rr[3];
        for (int k = 0; k < 3; ++k) {
            id3[k] = p->angles[3 * q + k];
            if (id3[k] < 0 || id3[k] >= h->N) { delete h; return MD_ERR_ARG; }
            rr[k] = 0;
            while (h->offsets[rr[k] + 1] <= id3[k]) ++rr[k];
        }
        if (id3[0] == id3[1] || id3[1] == id3[2] || id3[0] == id3[2] || rr[0] != rr[1] || rr[1] != rr[2]) {
            delete h;
            return MD_ERR_ARG;
        }
    }

    // list capacity: 1.5x the ideal-gas count in the list sphere at the
    // densest replica, plus a margin (grown on overflow by md_build_neighbors)
    if (p->list_capacity < 0) { delete h; return MD_ERR_ARG; }
    // a given capacity is rounded up to a multiple of 32 entries, like the
    // automatic one: every tile's list block then starts 64-byte aligned, as
    // the 16-byte copies of the list kernels require
    int K = (int)round_up(p->list_capacity, 32);
    h->auto_capacity = (K == 0);
    if (K == 0) {
        double kmax = 0;
        for (auto &R : h->reps) {
            double V = R.L[0] * R.L[1] * R.L[2];
            double rl = std::sqrt(R.rl2);
            kmax = std::fmax(kmax, 1.5 * (double)R.n / V * 4.18879020478639 * rl * rl * rl);
        }
        K = (int)round_up((long long)std::ceil(kmax) + 32, 32);
    }
    if (K > 65535) { delete h; return MD_ERR_ARG; }

    // halo capacity of the tile kernels, the largest over the replicas of: the
    // halo rows (3 x 3, fewer on axes of one or two cells), each holding a full
    // tile of kTileMax particles plus two cells at the mean occupancy, or the
    // whole row where that is less, with a margin; and never more than the
    // replica's particles, since a halo holds each of its cells once.  The
    // tiler keeps every halo within it (md_build_neighbors grows it when one
    // cell's halo alone does not fit), and a smaller capacity leaves room for
    // more blocks of the tile kernels per SM.
    double hneed = 0;
    for (auto &R : h->reps) {
        if (!R.ncells) continue;
        const double occ = (double)R.n / R.ncells;
        int ly, cy, lz, cz;
        mdk::axis_offsets(R.ncell[1], ly, cy);
        mdk::axis_offsets(R.ncell[2], lz, cz);
        const double row = std::fmin(R.ncell[0] * occ, mdk::kTileMax + 2.0 * occ) + 16.0;
        hneed = std::fmax(hneed, std::fmin((double)R.n, cy * cz * row));
    }
    int hcap = (int)round_up((long long)std::ceil(hneed), 128);
    hcap = std::min(std::max(hcap, 1024), 8192);

    Bufs &b = h->b;
    b.S = h->S;
    b.N = h->N;
    b.C = h->C;
    b.nrows = h->nrows;
    b.hcap = hcap;
    b.tile_max = mdk::kTileMax;
    b.nrep = nrep;
    b.nblk = h->nblk;
    b.dt = p->dt;
    b.mass = p->mass;
    b.half_dt_over_m = 0.5 * p->dt / p->mass;
    b.half_dt_over_m_fix = std::ldexp(b.half_dt_over_m, -22);
    b.gamma = p->langevin_gamma;
    b.kT = p->kT;
    b.langevin = p->langevin_gamma > 0 ? 1 : 0;
    b.noise_amp = b.langevin ? std::sqrt(24.0 * p->langevin_gamma * p->kT * p->mass / p->dt) : 0.0;
    b.seed = p->seed;
    b.fene_K = p->fene_K;
    b.fene_R02 = p->fene_R0 * p->fene_R0;
    b.fene_K_f = (float)p->fene_K;
    b.fene_R02_f = (float)(p->fene_R0 * p->fene_R0);

    bool ok = true;
    for (int q = 0; q < 2; ++q) {
        ok &= (b.x[q] = dalloc<double>(h, 3 * h->S)) != nullptr;
        ok &= (b.v[q] = dalloc<double>(h, 3 * h->S)) != nullptr;
        ok &= (b.pos[q] = dalloc<uint4>(h, h->S)) != nullptr;
    }
    ok &= (b.F = dalloc<double>(h, 3 * h->S)) != nullptr;
    ok &= (b.xref = dalloc<uint4>(h, h->S)) != nullptr;
    ok &= (b.slot_of_id = dalloc<int>(h, h->N)) != nullptr;
    ok &= (b.cellid = dalloc<int>(h, h->S)) != nullptr;
    ok &= (b.cell_count = dalloc<int>(h, h->C)) != nullptr;
    ok &= (b.cell_start = dalloc<int>(h, h->C)) != nullptr;
    ok &= (b.cell_end = dalloc<int>(h, h->C)) != nullptr;
    int *dpad = dalloc<int>(h, h->C);
    ok &= dpad != nullptr;
    ok &= (b.scan_part = dalloc<int>(h, (h->C + mdk::kScanBlock - 1) / mdk::kScanBlock + 1)) != nullptr;
    ok &= (b.bucket = dalloc<int>(h, h->S)) != nullptr;
    ok &= (b.nn = dalloc<int>(h, h->S)) != nullptr;
    ok &= (b.partial = dalloc<double>(h, 4 * (size_t)h->C)) != nullptr;
    ok &= (b.eacc = dalloc<long long>(h, 4 * (size_t)nrep)) != nullptr;
    ok &= (b.tiles = dalloc<mdk::Tile>(h, h->C)) != nullptr;
    ok &= (b.pieces = dalloc<mdk::Piece>(h, (size_t)h->C * (mdk::kMaxPieces + 1))) != nullptr;
    ok &= (b.tile_np = dalloc<int>(h, h->C)) != nullptr;
    ok &= (b.row_tiles = dalloc<int>(h, h->nrows + 1)) != nullptr;
    ok &= (b.rep_tile = dalloc<int>(h, nrep + 1)) != nullptr;
    ok &= (b.row_rep = dalloc<int>(h, h->nrows)) != nullptr;
    ok &= (b.ctl = dalloc<Ctl>(h, 1)) != nullptr;
    ok &= (h->stage = dalloc<double>(h, 6 * h->N)) != nullptr;
    ok &= (h->d_count = dalloc<unsigned long long>(h, 1)) != nullptr;
    Replica *drep = dalloc<Replica>(h, nrep);
    int *dblk = dalloc<int>(h, h->nblk);
    ok &= drep && dblk;
    if (!ok) { md_destroy(h); return MD_ERR_CUDA; }
    std::vector<int> blk(h->nblk, 0);
    for (int r = 0; r < nrep; ++r)
        for (int q = h->reps[r].blk_begin; q < h->reps[r].blk_end; ++q) blk[q] = r;
    std::vector<int> rowrep(h->nrows, 0);
    for (int r = 0; r < nrep; ++r)
        for (int q = 0; q < h->reps[r].ncell[1] * h->reps[r].ncell[2]; ++q) rowrep[h->reps[r].row_off + q] = r;
    ok &= cudaMemcpy(b.row_rep, rowrep.data(), sizeof(int) * h->nrows, cudaMemcpyHostToDevice) == cudaSuccess;
    // replica slot ranges are padded to kBlock: the padding follows the
    // replica's last cell in the scan, so the scan yields slot positions directly
    std::vector<int> pad(h->C, 0);
    for (int r = 0; r < nrep; ++r)
        if (h->reps[r].ncells > 0)
            pad[h->reps[r].cell_off + h->reps[r].ncells - 1] =
                (int)(round_up(h->reps[r].n, mdk::kBlock) - h->reps[r].n);
    ok &= cudaMemcpy(dpad, pad.data(), sizeof(int) * h->C, cudaMemcpyHostToDevice) == cudaSuccess;
    b.cell_pad = dpad;
    ok &= cudaMemcpy(drep, h->reps.data(), sizeof(Replica) * nrep, cudaMemcpyHostToDevice) == cudaSuccess;
    ok &= cudaMemcpy(dblk, blk.data(), sizeof(int) * h->nblk, cudaMemcpyHostToDevice) == cudaSuccess;
    ok &= cudaMemset(b.cell_count, 0, sizeof(int) * h->C) == cudaSuccess;
    ok &= cudaMemset(b.ctl, 0, sizeof(Ctl)) == cudaSuccess;
    ok &= cudaMemset(b.eacc, 0, sizeof(long long) * 4 * (size_t)nrep) == cudaSuccess;
    b.rep = drep;
    b.blk_rep = dblk;

    // FENE bonds as a per-particle adjacency (both directions)
    if (p->n_bonds > 0) {
        std::vector<int> deg(h->N + 1, 0);
        for (int64_t q = 0; q < p->n_bonds; ++q) {
            long long a = p->bonds[2 * q], c = p->bonds[2 * q + 1];
            deg[a + 1]++;
            deg[c + 1]++;
        }
        for (long long q = 0; q < h->N; ++q) deg[q + 1] += deg[q];
        std::vector<int> partner(2 * p->n_bonds);
        std::vector<int> fill(deg.begin(), deg.end() - 1);
        for (int64_t q = 0; q < p->n_bonds; ++q) {
            int a = p->bonds[2 * q], c = p->bonds[2 * q + 1];
            partner[fill[a]++] = c;
            partner[fill[c]++] = a;
        }
        int *doff = dalloc<int>(h, h->N + 1);
        int *dpart = dalloc<int>(h, partner.size());
        if (!doff || !dpart) { md_destroy(h); return MD_ERR_CUDA; }
        ok &= cudaMemcpy(doff, deg.data(), sizeof(int) * (h->N + 1), cudaMemcpyHostToDevice) == cudaSuccess;
        ok &= cudaMemcpy(dpart, partner.data(), sizeof(int) * partner.size(), cudaMemcpyHostToDevice) == cudaSuccess;
        b.bond_off = doff;
        b.n_bond_ent = (long long)partner.size();
        if (!(b.bond_pslot = dalloc<int>(h, partner.size()))) { md_destroy(h); return MD_ERR_CUDA; }
        b.bond_partner = dpart;
        b.has_bonds = 1;
    }
    // angle triples as a per-particle list: every particle of a triple gets the
    // whole triple and its role in it
    if (p->n_angles > 0) {
        std::vector<int> deg(h->N + 1, 0);
        for (int64_t q = 0; q < p->n_angles; ++q)
            for (int k = 0; k < 3; ++k) deg[p->angles[3 * q + k] + 1]++;
        for (long long q = 0; q < h->N; ++q) deg[q + 1] += deg[q];
        std::vector<int4> ent(3 * p->n_angles);
        std::vector<int> fill(deg.begin(), deg.end() - 1);
        for (int64_t q = 0; q < p->n_angles; ++q)
            for (int k = 0; k < 3; ++k)
                ent[fill[p->angles[3 * q + k]]++] =
                    make_int4(p->angles[3 * q], p->angles[3 * q + 1], p->angles[3 * q + 2], k);
        int *doff = dalloc<int>(h, h->N + 1);
        int4 *dent = dalloc<int4>(h, ent.size());
        if (!doff || !dent) { md_destroy(h); return MD_ERR_CUDA; }
        ok &= cudaMemcpy(doff, deg.data(), sizeof(int) * (h->N + 1), cudaMemcpyHostToDevice) == cudaSuccess;
        ok &= cudaMemcpy(dent, ent.data(), sizeof(int4) * ent.size(), cudaMemcpyHostToDevice) == cudaSuccess;
        b.ang_off = doff;
        b.ang_ent = dent;
        b.n_ang_ent = (long long)ent.size();
        if (!(b.ang_slot = dalloc<int4>(h, ent.size()))) { md_destroy(h); return MD_ERR_CUDA; }
        b.has_angles = 1;
        b.angle_K = p->angle_K;
        b.angle_K_f = (float)p->angle_K;
    }
    if (!ok) { md_destroy(h); return MD_ERR_CUDA; }
    if (alloc_list(h, K) != MD_OK) { md_destroy(h); return MD_ERR_CUDA; }
    *out = h;
    return MD_OK;
}

void md_destroy(md_handle *h)
{
    if (!h) return;
    cudaDeviceSynchronize();
    for (void *q : h->allocs) cudaFree(q);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    if (h->gexec_e) cudaGraphExecDestroy(h->gexec_e);
    if (h->graph_e) cudaGraphDestroy(h->graph_e);
    if (h->gexec_chain) cudaGraphExecDestroy(h->gexec_chain);
    if (h->graph_chain) cudaGraphDestroy(h->graph_chain);
    if (h->gexec_x) cudaGraphExecDestroy(h->gexec_x);
    if (h->graph_x) cudaGraphDestroy(h->graph_x);
    if (h->cap) cudaStreamDestroy(h->cap);
    delete h;
}

md_status md_set_state(md_handle *h, const double *x, const double *v, void *stream)
{
    if (!h || !x || !v) return fail(h, MD_ERR_ARG, "md_set_state: null argument");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = sizeof(double) * 3 * (size_t)h->N;
    double *xs = h->stage, *vs = h->stage + 3 * h->N;
    if (!cuda_ok(h, cudaMemcpyAsync(xs, x, bytes, cudaMemcpyDefault, st), "copy positions") ||
        !cuda_ok(h, cudaMemcpyAsync(vs, v, bytes, cudaMemcpyDefault, st), "copy velocities") ||
        !cuda_ok(h, cudaMemsetAsync(h->b.cell_count, 0, sizeof(int) * h->C, st), "clear cells"))
        return MD_ERR_CUDA;
    // a launch cut short by a latched error can leave sums behind
    if (h->b.Fq && !cuda_ok(h, cudaMemsetAsync(h->b.Fq, 0, sizeof(long long) * 3 * h->S, st), "clear force sums"))
        return MD_ERR_CUDA;
    if (!cuda_ok(h, cudaMemsetAsync(h->b.eacc, 0, sizeof(long long) * 4 * (size_t)h->b.nrep, st), "clear energy sums"))
        return MD_ERR_CUDA;
    mdk::launch_set_state(h->b, xs, vs, st);
    if (!cuda_ok(h, cudaGetLastError(), "set_state launch")) return MD_ERR_CUDA;
    h->state_set = true;
    h->F_valid = false;
    h->built = false;
    return MD_OK;
}

// With an automatic list capacity, the first list of a new state is built by
// md_build_neighbors, which grows the capacity until the list fits (the
// capacity is first sized from the mean density, which an uneven system such
// as a liquid/vapour slab exceeds).  One synchronisation per md_set_state.
static md_status first_build(md_handle *h, void *stream)
{
    if (!h->auto_capacity || h->built) return MD_OK;
    return md_build_neighbors(h, stream);
}

md_status md_get_state(md_handle *h, double *x, double *v, void *stream)
{
    if (!h) return MD_ERR_ARG;
    if (!h->state_set) return fail(h, MD_ERR_ARG, "md_get_state before md_set_state");
    cudaStream_t st = (cudaStream_t)stream;
    double *xs = h->stage, *vs = h->stage + 3 * h->N;
    mdk::launch_get_state(h->b, x ? xs : nullptr, v ? vs : nullptr, st);
    const size_t bytes = sizeof(double) * 3 * (size_t)h->N;
    if (x && !cuda_ok(h, cudaMemcpyAsync(x, xs, bytes, cudaMemcpyDefault, st), "copy positions out"))
        return MD_ERR_CUDA;
    if (v && !cuda_ok(h, cudaMemcpyAsync(v, vs, bytes, cudaMemcpyDefault, st), "copy velocities out"))
        return MD_ERR_CUDA;
    return sync_and_check(h, st);
}

md_status md_get_checkpoint(md_handle *h, double *x, double *v, double *f, int64_t *step, void *stream)
{
    if (!h || !x || !v || !f || !step) return fail(h, MD_ERR_ARG, "md_get_checkpoint: null argument");
    if (!h->state_set) return fail(h, MD_ERR_ARG, "md_get_checkpoint before md_set_state");
    cudaStream_t st = (cudaStream_t)stream;
    // the force the next step starts from; evaluated now, as md_step would,
    // when none is stored
    md_status s0 = first_build(h, stream);
    if (s0 != MD_OK) return s0;
    if (!h->F_valid) {
        mdk::launch_rebuild_chain(h->b, st);
        mdk::launch_force(h->b, h->precision, mdk::kModeStore, false, st);
        if (!cuda_ok(h, cudaGetLastError(), "force launch")) return MD_ERR_CUDA;
        h->F_valid = true;
    }
    double *xs = h->stage, *vs = h->stage + 3 * h->N;
    const size_t bytes = sizeof(double) * 3 * (size_t)h->N;
    mdk::launch_get_state(h->b, xs, vs, st);
    if (!cuda_ok(h, cudaMemcpyAsync(x, xs, bytes, cudaMemcpyDefault, st), "copy positions out") ||
        !cuda_ok(h, cudaMemcpyAsync(v, vs, bytes, cudaMemcpyDefault, st), "copy velocities out"))
        return MD_ERR_CUDA;
    mdk::launch_force_by_id(h->b, xs, 0, st);
    if (!cuda_ok(h, cudaMemcpyAsync(f, xs, bytes, cudaMemcpyDefault, st), "copy force out")) return MD_ERR_CUDA;
    md_status s = sync_and_check(h, st);
    if (s != MD_OK) return s;
    Ctl c;
    if ((s = read_ctl(h, &c)) != MD_OK) return s;
    *step = (int64_t)c.step;
    return MD_OK;
}

md_status md_set_checkpoint(md_handle *h, const double *x, const double *v, const double *f, int64_t step,
                            void *stream)
{
    if (!h || !x || !v || !f || step < 0) return fail(h, MD_ERR_ARG, "md_set_checkpoint: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    md_status s = md_set_state(h, x, v, stream);
    if (s != MD_OK) return s;
    // the step counter keys the Langevin noise: the resumed run draws the
    // numbers the uninterrupted one would have drawn
    const long long stp = (long long)step;
    if (!cuda_ok(h, cudaMemcpyAsync(&h->b.ctl->step, &stp, sizeof(long long), cudaMemcpyHostToDevice, st),
                 "restore step"))
        return MD_ERR_CUDA;
    // sort and build the list now (growing an automatic capacity as needed),
    // then put the stored force into the particles' new slots (the copy goes
    // through the handle's staging buffer)
    s = md_build_neighbors(h, stream);
    if (s != MD_OK) return s;
    double *fs = h->stage;
    if (!cuda_ok(h, cudaMemcpyAsync(fs, f, sizeof(double) * 3 * (size_t)h->N, cudaMemcpyDefault, st), "copy force in"))
        return MD_ERR_CUDA;
    mdk::launch_force_by_id(h->b, fs, 1, st);
    if (!cuda_ok(h, cudaGetLastError(), "checkpoint launch")) return MD_ERR_CUDA;
    s = sync_and_check(h, st);
    if (s != MD_OK) return s;
    h->F_valid = true;
    return MD_OK;
}

md_status md_build_neighbors(md_handle *h, void *stream)
{
    if (!h) return MD_ERR_ARG;
    if (!h->state_set) return fail(h, MD_ERR_ARG, "md_build_neighbors before md_set_state");
    cudaStream_t st = (cudaStream_t)stream;
    mdk::launch_set_rebuild(h->b, st);
    mdk::launch_rebuild_chain(h->b, st);
    h->F_valid = false;
    if (!cuda_ok(h, cudaGetLastError(), "rebuild launch")) return MD_ERR_CUDA;
    if (!h->auto_capacity) return MD_OK;
    // automatic capacity: check the build and grow the list if it overflowed
    Ctl c;
    if (!cuda_ok(h, cudaStreamSynchronize(st), "stream synchronize")) return MD_ERR_CUDA;
    if (read_ctl(h, &c) != MD_OK) return MD_ERR_CUDA;
    if ((c.err & mdk::kErrList) && c.err == mdk::kErrList) {
        md_status g = grow_after_overflow(h, c);
        if (g != MD_OK) return g;
        // the overflowing build still sorted the state; build again with the larger capacities
        mdk::launch_set_rebuild(h->b, st);
        mdk::launch_rebuild_chain(h->b, st);
        const md_status s2 = sync_and_check(h, st);
        if (s2 == MD_OK) h->built = true;
        return s2;
    }
    const md_status s1 = status_of(h, c);
    if (s1 == MD_OK) h->built = true;
    return s1;
}

md_status md_compute_forces(md_handle *h, double *f_out, double *euw_out, void *stream)
{
    if (!h) return MD_ERR_ARG;
    if (!h->state_set) return fail(h, MD_ERR_ARG, "md_compute_forces before md_set_state");
    md_status s0 = first_build(h, stream);
    if (s0 != MD_OK) return s0;
    cudaStream_t st = (cudaStream_t)stream;
    mdk::launch_rebuild_chain(h->b, st);
    h->F_valid = false;
    Bufs b = h->b;
    double *fs = h->stage;   // 3 N
    double *th = nullptr;
    if (euw_out) {
        if (ensure_thermo(h, 3LL * h->b.nrep) != MD_OK) return MD_ERR_CUDA;
        th = h->thermo_stage;
    }
    b.fout = f_out ? fs : nullptr;
    b.thermo = euw_out ? th : nullptr;
    mdk::launch_force(b, h->precision, mdk::kModeOut, euw_out != nullptr, st);
    if (!cuda_ok(h, cudaGetLastError(), "force launch")) return MD_ERR_CUDA;
    if (f_out && !cuda_ok(h, cudaMemcpyAsync(f_out, fs, sizeof(double) * 3 * h->N, cudaMemcpyDefault, st),
                          "copy forces out"))
        return MD_ERR_CUDA;
    if (euw_out && !cuda_ok(h, cudaMemcpyAsync(euw_out, th, sizeof(double) * 3 * h->b.nrep, cudaMemcpyDefault, st),
                            "copy energies out"))
        return MD_ERR_CUDA;
    return MD_OK;
}

}  // extern "C"

// The kernel sequence of md_step (asynchronous).
static md_status step_launch(md_handle *h, int32_t nsteps, int32_t thermo_every, double *thermo_out, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    const int nrep = h->b.nrep;
    const long long nrec = thermo_every > 0 ? nsteps / thermo_every : 0;
    if (nrec > 0 && ensure_thermo(h, nrec * 3 * nrep) != MD_OK) return MD_ERR_CUDA;
    Bufs b = h->b;
    const bool every = nrec > 0 && thermo_every == 1;
    if (!h->timing && (nrec == 0 || every) && h->use_graph && build_step_graph(h, every)) {
        if (!h->F_valid) {
            mdk::launch_rebuild_chain(b, st);
            mdk::launch_force(b, h->precision, mdk::kModeStore, false, st);
        }
        mdk::launch_set_steps(b, (long long)nsteps - 1, st);
        if (!cuda_ok(h, cudaGraphLaunch(every ? h->gexec_e : h->gexec, st), "graph launch")) return MD_ERR_CUDA;
        h->F_valid = true;
        if (every &&
            !cuda_ok(h, cudaMemcpyAsync(thermo_out, h->thermo_stage, sizeof(double) * nrec * 3 * nrep,
                                        cudaMemcpyDefault, st), "copy thermo out"))
            return MD_ERR_CUDA;
        return MD_OK;
    }
    cudaGetLastError();   // a failed graph build leaves nothing behind: fall back to stream launches
    if (h->timing && h->ev_marks.size() > 100000) resolve_timing(h);   // bounded event pool
    long long t0 = mark(h, st);
    if (!h->F_valid) {
        mdk::launch_rebuild_chain(b, st);
        mdk::launch_force(b, h->precision, mdk::kModeStore, false, st);
    }
    mdk::launch_kick_drift(b, st);
    section(h, MD_SECT_OTHER, t0, mark(h, st));
    for (int t = 1; t <= nsteps; ++t) {
        const bool rec = thermo_every > 0 && (t % thermo_every) == 0;
        b.thermo = rec ? h->thermo_stage + (long long)(t / thermo_every - 1) * 3 * nrep : nullptr;
        long long a = mark(h, st);
        mdk::launch_rebuild_chain(b, st);
        long long m = mark(h, st);
        mdk::launch_force(b, h->precision, t < nsteps ? mdk::kModeFused : mdk::kModeFinal, rec, st);
        long long e = mark(h, st);
        section(h, MD_SECT_NEIGH, a, m);
        section(h, t < nsteps ? MD_SECT_FORCE : MD_SECT_OTHER, m, e);
    }
    if (!cuda_ok(h, cudaGetLastError(), "step launch")) return MD_ERR_CUDA;
    h->F_valid = true;
    if (nrec > 0 &&
        !cuda_ok(h, cudaMemcpyAsync(thermo_out, h->thermo_stage, sizeof(double) * nrec * 3 * nrep, cudaMemcpyDefault, st),
                 "copy thermo out"))
        return MD_ERR_CUDA;
    return MD_OK;
}

// The rest of an md_step call after an overflowing rebuild: the state holds
// x at the step t_start of the call (counted from its start) and the
// half-step velocity before it, its force not yet evaluated.  Rebuilds the
// list there, then runs the fused force + update of steps t_start ..
// nsteps - 1 and the final force, with their energy records in place.
static md_status step_resume(md_handle *h, int t_start, int32_t nsteps, int32_t thermo_every, cudaStream_t st)
{
    Bufs b = h->b;
    const int nrep = b.nrep;
    mdk::launch_set_rebuild(b, st);
    for (int t = t_start; t <= nsteps; ++t) {
        const bool rec = thermo_every > 0 && (t % thermo_every) == 0;
        b.thermo = rec ? h->thermo_stage + (long long)(t / thermo_every - 1) * 3 * nrep : nullptr;
        mdk::launch_rebuild_chain(b, st);
        mdk::launch_force(b, h->precision, t < nsteps ? mdk::kModeFused : mdk::kModeFinal, rec, st);
    }
    return cuda_ok(h, cudaGetLastError(), "step launch") ? MD_OK : MD_ERR_CUDA;
}

extern "C" {

md_status md_step(md_handle *h, int32_t nsteps, int32_t thermo_every, double *thermo_out, void *stream)
{
    if (!h || nsteps < 0 || thermo_every < 0 || (thermo_every > 0 && !thermo_out))
        return fail(h, MD_ERR_ARG, "md_step: bad arguments");
    if (!h->state_set) return fail(h, MD_ERR_ARG, "md_step before md_set_state");
    if (nsteps == 0) return MD_OK;
    md_status s0 = first_build(h, stream);
    if (s0 != MD_OK) return s0;
    if (!h->recover) return step_launch(h, nsteps, thermo_every, thermo_out, stream);
    // recovery: the step counter at the start of the call, then the call,
    // then (after a list or halo overflow) growth and the rest of the call
    cudaStream_t st = (cudaStream_t)stream;
    md_status s = sync_and_check(h, st);
    if (s != MD_OK) return s;
    Ctl c;
    if ((s = read_ctl(h, &c)) != MD_OK) return s;
    const long long step0 = c.step;
    s = step_launch(h, nsteps, thermo_every, thermo_out, stream);
    if (s != MD_OK) return s;
    for (int attempt = 0;; ++attempt) {
        if (!cuda_ok(h, cudaStreamSynchronize(st), "stream synchronize")) return MD_ERR_CUDA;
        if ((s = read_ctl(h, &c)) != MD_OK) return s;
        if (c.err != mdk::kErrList || attempt == 4) return status_of(h, c);
        if ((s = grow_after_overflow(h, c)) != MD_OK) return s;
        h->recoveries += 1;
        const long long done = c.step - step0;   // drifts completed before the failing rebuild
        if (done <= 0) {
            // the rebuild before the first drift failed: the whole call again
            // (that build cleared the rebuild flag, so it is set again)
            mdk::launch_set_rebuild(h->b, st);
            h->F_valid = false;
            s = step_launch(h, nsteps, thermo_every, thermo_out, stream);
        } else {
            s = step_resume(h, (int)done, nsteps, thermo_every, st);
            const long long nrec = thermo_every > 0 ? nsteps / thermo_every : 0;
            if (s == MD_OK && nrec > 0 &&
                !cuda_ok(h, cudaMemcpyAsync(thermo_out, h->thermo_stage, sizeof(double) * nrec * 3 * h->b.nrep,
                                            cudaMemcpyDefault, st), "copy thermo out"))
                s = MD_ERR_CUDA;
            h->F_valid = true;
        }
        if (s != MD_OK) return s;
    }
}

md_status md_check_wait_timeout(md_handle *h, int32_t polls, void *stream)
{
    if (!h) return MD_ERR_ARG;
    if (polls < 1 || polls > 65536) return fail(h, MD_ERR_ARG, "md_check_wait_timeout: polls outside 1..65536");
    mdk::launch_wait_selftest(h->b, polls, (cudaStream_t)stream);
    return cuda_ok(h, cudaGetLastError(), "self-test launch") ? MD_OK : MD_ERR_CUDA;
}

int md_build_flags(void)
{
    return mdk::kChecked ? MD_BUILD_CHECKED : 0;
}

md_status md_check_bounds_selftest(md_handle *h, int32_t site, void *stream)
{
    if (!h) return MD_ERR_ARG;
    if (!mdk::kChecked) return fail(h, MD_ERR_ARG, "md_check_bounds_selftest: not a checked build (MD_CHECKED)");
    if (site < 0 || site >= mdk::kSiteCount) return fail(h, MD_ERR_ARG, "md_check_bounds_selftest: site out of range");
    const int v = site;
    return cuda_ok(h, cudaMemcpyAsync(&h->b.ctl->plant, &v, sizeof(int), cudaMemcpyHostToDevice, (cudaStream_t)stream),
                   "arm bounds self-test") &&
                   cuda_ok(h, cudaStreamSynchronize((cudaStream_t)stream), "arm bounds self-test")
               ? MD_OK
               : MD_ERR_CUDA;
}

md_status md_set_recovery(md_handle *h, int32_t enable)
{
    if (!h) return MD_ERR_ARG;
    h->recover = enable != 0;
    return MD_OK;
}

md_status md_export_pairs(md_handle *h, int32_t *pairs_out, int64_t capacity, int64_t *n_out, void *stream)
{
    if (!h || !n_out || capacity < 0 || (capacity > 0 && !pairs_out)) return fail(h, MD_ERR_ARG, "md_export_pairs: bad arguments");
    if (!h->state_set) return fail(h, MD_ERR_ARG, "md_export_pairs before md_set_state");
    cudaStream_t st = (cudaStream_t)stream;
    md_status s = sync_and_check(h, st);
    if (s != MD_OK) return s;
    int *tmp = nullptr;
    if (capacity > 0 && !cuda_ok(h, cudaMalloc(&tmp, sizeof(int) * 2 * (size_t)capacity), "pair buffer"))
        return MD_ERR_CUDA;
    cudaMemsetAsync(h->d_count, 0, sizeof(unsigned long long), st);
    mdk::launch_export_pairs(h->b, tmp, capacity, h->d_count, st);
    unsigned long long cnt = 0;
    bool ok = cuda_ok(h, cudaMemcpyAsync(&cnt, h->d_count, sizeof(cnt), cudaMemcpyDeviceToHost, st), "pair count") &&
              cuda_ok(h, cudaStreamSynchronize(st), "stream synchronize");
    if (ok && capacity > 0) {
        long long m = (long long)cnt < capacity ? (long long)cnt : capacity;
        ok = cuda_ok(h, cudaMemcpy(pairs_out, tmp, sizeof(int) * 2 * (size_t)m, cudaMemcpyDefault), "copy pairs out");
    }
    if (tmp) cudaFree(tmp);
    if (!ok) return MD_ERR_CUDA;
    *n_out = (int64_t)cnt;
    return MD_OK;
}

md_status md_sync(md_handle *h, void *stream)
{
    if (!h) return MD_ERR_ARG;
    return sync_and_check(h, (cudaStream_t)stream);
}

md_status md_get_stats(md_handle *h, md_stats *out)
{
    if (!h || !out) return MD_ERR_ARG;
    if (!cuda_ok(h, cudaDeviceSynchronize(), "device synchronize")) return MD_ERR_CUDA;
    Ctl c;
    md_status s = read_ctl(h, &c);
    if (s != MD_OK) return s;
    std::memset(out, 0, sizeof(*out));
    out->steps = c.step;
    out->rebuilds = c.rebuilds;
    out->list_entries = c.list_entries;
    out->max_list_len = c.max_nn;
    out->list_capacity = h->K;
    out->max_cell_occupancy = c.max_occ;
    out->error_word = c.err;
    for (int k = 0; k < 3; ++k) out->ncell[k] = h->reps[0].ncell[k];
    out->n_replicas = h->b.nrep;
    out->n_particles = h->N;
    out->n_tiles = c.ntiles;
    out->max_halo = c.max_halo;
    out->halo_capacity = h->b.hcap;
    out->tile_size = h->b.tile_max;
    out->recoveries = h->recoveries;
    out->bad_site = c.bad_site;
    out->bad_index = c.bad_index;
    return status_of(h, c);
}

md_status md_forward(md_handle *h, int32_t nsteps, int32_t ckpt_every, double *euw_out, void *stream)
{
    if (!h || nsteps < 0 || ckpt_every < 1) return fail(h, MD_ERR_ARG, "md_forward: bad arguments");
    if (!h->state_set) return fail(h, MD_ERR_ARG, "md_forward before md_set_state");
    if (h->b.has_bonds || h->b.has_angles || h->b.langevin || h->p.potential == MD_SOFT)
        return fail(h, MD_ERR_ARG, "md_forward: the adjoint covers NVE LJ / WCA pair forces only (no bonds, angles, thermostat or push-off)");
    if (h->b.half_list) return fail(h, MD_ERR_ARG, "md_forward: the adjoint walks the full list (md_set_half_list(h, 0))");
    cudaStream_t st = (cudaStream_t)stream;
    const long long n6 = 6LL * h->N;
    const long long nck = nsteps / ckpt_every + 1;
    if (h->ad_ck_cap < nck) {
        h->ad_ck = grow(h, h->ad_ck, (size_t)(nck * n6));
        if (!h->ad_ck) return fail(h, MD_ERR_CUDA, "cannot allocate checkpoints");
        h->ad_ck_cap = nck;
    }
    if (!h->ad_fin && !(h->ad_fin = dalloc<double>(h, (size_t)n6))) return fail(h, MD_ERR_CUDA, "cannot allocate");
    h->ad_ready = false;
    for (long long c = 0; c < nck; ++c) {
        double *ck = h->ad_ck + c * n6;
        mdk::launch_get_state(h->b, ck, ck + 3 * h->N, st);
        const long long rest = nsteps - c * ckpt_every;
        const int run = (int)std::min<long long>(ckpt_every, rest);
        if (run > 0) {
            md_status s = md_step(h, run, 0, nullptr, stream);
            if (s != MD_OK) return s;
        }
    }
    mdk::launch_get_state(h->b, h->ad_fin, h->ad_fin + 3 * h->N, st);
    if (euw_out) {
        md_status s = md_compute_forces(h, nullptr, euw_out, stream);
        if (s != MD_OK) return s;
    }
    h->ad_T = nsteps;
    h->ad_k = ckpt_every;
    md_status s = sync_and_check(h, st);
    if (s == MD_OK) h->ad_ready = true;
    return s;
}

// set the handle's state from caller-order device arrays and build its lists
// Positions x (caller order, device) into the particles' current slots; the
// Verlet list is rebuilt only if the displacement since its build asks for it.
// The steps of a checkpoint segment again, with the positions after each
// step in slots 1..nsteps of ad_seg: one graph launch of md_step's loop with a
// recording node after every drift (step by step with section timers, without
// graphs, or with overflow recovery, whose md_step calls synchronise).
static md_status step_record(md_handle *h, int nsteps, cudaStream_t st)
{
    if (nsteps <= 0) return MD_OK;
    md_status s = first_build(h, st);
    if (s != MD_OK) return s;
    const long long n3 = 3 * h->N;
    if (!h->timing && !h->recover && h->use_graph && build_step_graph(h, false, true)) {
        Bufs b = h->b;
        if (!h->F_valid) {
            mdk::launch_rebuild_chain(b, st);
            mdk::launch_force(b, h->precision, mdk::kModeStore, false, st);
        }
        mdk::launch_set_steps(b, (long long)nsteps - 1, st);
        if (!cuda_ok(h, cudaGraphLaunch(h->gexec_x, st), "graph launch")) return MD_ERR_CUDA;
        h->F_valid = true;
        return MD_OK;
    }
    cudaGetLastError();   // a failed graph build leaves nothing behind
    for (int t = 1; t <= nsteps; ++t) {
        s = md_step(h, 1, 0, nullptr, st);
        if (s != MD_OK) return s;
        mdk::launch_get_state(h->b, h->ad_seg + (long long)t * n3, nullptr, st);
    }
    return MD_OK;
}

static md_status adj_load(md_handle *h, const double *x, cudaStream_t st)
{
    mdk::launch_reload(h->b, x, st);
    if (!h->timing && h->use_graph && build_chain_graph(h)) {
        if (!cuda_ok(h, cudaGraphLaunch(h->gexec_chain, st), "graph launch")) return MD_ERR_CUDA;
    } else {
        cudaGetLastError();   // a failed graph build leaves nothing behind: stream launches
        mdk::launch_rebuild_chain(h->b, st);
    }
    h->F_valid = false;
    return cuda_ok(h, cudaGetLastError(), "reload launch") ? MD_OK : MD_ERR_CUDA;
}

md_status md_backward(md_handle *h, const double *dL_dx, const double *dL_dv, const double *dL_deuw, double *dL_deps,
                      double *dL_dsigma, void *stream)
{
    if (!h || !dL_deps || !dL_dsigma) return fail(h, MD_ERR_ARG, "md_backward: null argument");
    if (!h->ad_ready) return fail(h, MD_ERR_ARG, "md_backward without a recorded md_forward");
    cudaStream_t st = (cudaStream_t)stream;
    const int nrep = h->b.nrep;
    const long long N = h->N, n3 = 3 * N;
    const int T = h->ad_T, k = h->ad_k;
    if (!h->ad_work && !(h->ad_work = dalloc<double>(h, (size_t)(3 * n3)))) return fail(h, MD_ERR_CUDA, "cannot allocate");
    if (h->ad_seg_cap < k + 1) {
        h->ad_seg = grow(h, h->ad_seg, (size_t)((k + 1) * n3));
        if (!h->ad_seg) return fail(h, MD_ERR_CUDA, "cannot allocate");
        h->ad_seg_cap = k + 1;
        h->gen++;   // the recording step graph holds the buffer's address
    }
    if (!h->ad_small && !(h->ad_small = dalloc<double>(h, (size_t)(12 * nrep)))) return fail(h, MD_ERR_CUDA, "cannot allocate");
    if (h->precision == MD_FP32_FIXED && !h->b.adj_wa) {
        h->b.adj_wa = dalloc<float4>(h, (size_t)h->S);
        h->b.adj_wb = dalloc<float2>(h, (size_t)h->S);
        if (!h->b.adj_wa || !h->b.adj_wb) return fail(h, MD_ERR_CUDA, "cannot allocate");
    }
    double *lx = h->ad_work, *lv = lx + n3, *hv = lv + n3;
    double *coef = h->ad_small, *g = coef + 4 * nrep, *sums = g + 4 * nrep;
    // loss weights (dL/dU, dL/dK, dL/dW) per replica, from host or device memory
    std::vector<double> in(3 * nrep, 0.0), cf(12 * nrep, 0.0);
    if (dL_deuw &&
        !cuda_ok(h, cudaMemcpy(in.data(), dL_deuw, sizeof(double) * 3 * nrep, cudaMemcpyDefault), "read dL_deuw"))
        return MD_ERR_CUDA;
    for (int r = 0; r < nrep; ++r)
        for (int q = 0; q < 3; ++q) cf[4 * r + q] = in[3 * r + q];
    if (!cuda_ok(h, cudaMemcpyAsync(coef, cf.data(), sizeof(double) * 12 * nrep, cudaMemcpyHostToDevice, st), "upload"))
        return MD_ERR_CUDA;
    const double half = 0.5 * h->b.dt / h->b.mass;
    // final state: adjoints of the loss and its explicit parameter terms
    md_status s = adj_load(h, h->ad_fin, st);
    if (s != MD_OK) return s;
    mdk::launch_adj_loss(h->b, coef, lx, lv, sums, st);
    mdk::launch_adj_finish_loss(h->b, sums, coef, g, st);
    // the loss's own gradients in the final positions and velocities join
    // the terminal adjoints (staged through the handle's buffer: they may be
    // host memory)
    if (dL_dx || dL_dv) {
        double *gx = h->stage, *gv = h->stage + n3;
        if (dL_dx && !cuda_ok(h, cudaMemcpyAsync(gx, dL_dx, sizeof(double) * n3, cudaMemcpyDefault, st), "read dL_dx"))
            return MD_ERR_CUDA;
        if (dL_dv && !cuda_ok(h, cudaMemcpyAsync(gv, dL_dv, sizeof(double) * n3, cudaMemcpyDefault, st), "read dL_dv"))
            return MD_ERR_CUDA;
        mdk::launch_adj_add(n3, lx, lv, dL_dx ? gx : nullptr, dL_dv ? gv : nullptr, st);
    }
    // reverse through the steps, one checkpoint segment at a time (last first)
    if (T > 0) {
        const int nseg = (T + k - 1) / k;
        for (int c = nseg - 1; c >= 0; --c) {
            const int t0 = c * k, t1 = std::min(T, (c + 1) * k);
            const double *ck = h->ad_ck + (long long)c * 2 * n3;
            // an error latched by the reverse pass so far is reported before
            // md_set_state clears the error word for the segment's re-run
            s = sync_and_check(h, st);
            if (s != MD_OK) return s;
            s = md_set_state(h, ck, ck + n3, st);
            if (s != MD_OK) return s;
            if (!cuda_ok(h, cudaMemcpyAsync(h->ad_seg, ck, sizeof(double) * n3, cudaMemcpyDeviceToDevice, st), "copy"))
                return MD_ERR_CUDA;
            s = step_record(h, t1 - t0, st);
            if (s != MD_OK) return s;
            for (int t = t1; t >= (c == 0 ? 0 : t0 + 1); --t) {
                s = adj_load(h, h->ad_seg + (long long)(t - t0) * n3, st);
                if (s != MD_OK) return s;
                // the kicks at x_t: the first half kick of step t and the second of step t - 1
                const double ct = (t == T || t == 0) ? half : 2.0 * half;
                mdk::launch_adj_hvp(h->b, h->precision, lv, hv, ct, g, st);
                mdk::launch_adj_update(n3, lx, lv, hv, ct, t > 0 ? h->b.dt : 0.0, st);
            }
        }
    }
    std::vector<double> gh(4 * nrep), ge(nrep), gs(nrep);
    if (!cuda_ok(h, cudaMemcpyAsync(gh.data(), g, sizeof(double) * 4 * nrep, cudaMemcpyDeviceToHost, st), "read g"))
        return MD_ERR_CUDA;
    s = sync_and_check(h, st);
    if (s != MD_OK) return s;
    for (int r = 0; r < nrep; ++r) { ge[r] = gh[4 * r]; gs[r] = gh[4 * r + 1]; }
    if (!cuda_ok(h, cudaMemcpy(dL_deps, ge.data(), sizeof(double) * nrep, cudaMemcpyDefault), "write dL_deps") ||
        !cuda_ok(h, cudaMemcpy(dL_dsigma, gs.data(), sizeof(double) * nrep, cudaMemcpyDefault), "write dL_dsigma"))
        return MD_ERR_CUDA;
    // leave the handle at the final state of the recorded run
    s = md_set_state(h, h->ad_fin, h->ad_fin + n3, st);
    if (s != MD_OK) return s;
    return sync_and_check(h, st);
}

md_status md_set_half_list(md_handle *h, int32_t enable, void *stream)
{
    if (!h) return MD_ERR_ARG;
    const int want = enable ? 1 : 0;
    if (want == h->b.half_list) return MD_OK;
    if (want && h->precision != MD_FP32_FIXED)
        return fail(h, MD_ERR_ARG, "md_set_half_list: the half list needs MD_FP32_FIXED");
    if (want && (h->b.has_bonds || h->b.has_angles))
        return fail(h, MD_ERR_ARG, "md_set_half_list: the half list covers pair forces without bonds or angles");
    cudaStream_t st = (cudaStream_t)stream;
    if (want && !h->b.Fq) {
        h->b.Fq = dalloc<long long>(h, 3 * (size_t)h->S);
        if (!h->b.Fq) return fail(h, MD_ERR_CUDA, "cannot allocate the fixed-point force sums");
        if (!cuda_ok(h, cudaMemsetAsync(h->b.Fq, 0, sizeof(long long) * 3 * h->S, st), "clear force sums"))
            return MD_ERR_CUDA;
    }
    h->b.half_list = want;
    h->gen++;             // the step graph holds the old Bufs by value
    h->ad_ready = false;
    // the next call must rebuild before any force: md_step then starts from
    // a fresh force evaluation instead of the stored one (the same values),
    // so its first drift cannot clear the pending rebuild
    h->F_valid = false;
    if (h->state_set) {   // the next step, force or list call rebuilds the list in the new form
        mdk::launch_set_rebuild(h->b, st);
        if (!cuda_ok(h, cudaGetLastError(), "set_rebuild launch")) return MD_ERR_CUDA;
    }
    return MD_OK;
}

md_status md_set_tile_size(md_handle *h, int32_t tile_size, void *stream)
{
    if (!h) return MD_ERR_ARG;
    if (tile_size < 1 || tile_size > mdk::kTileMax) return fail(h, MD_ERR_ARG, "md_set_tile_size: size outside 1..128");
    if (tile_size == h->b.tile_max) return MD_OK;
    h->b.tile_max = tile_size;
    h->gen++;   // the step graph holds the old Bufs by value
    if (h->state_set) {
        mdk::launch_set_rebuild(h->b, (cudaStream_t)stream);
        if (!cuda_ok(h, cudaGetLastError(), "set_rebuild launch")) return MD_ERR_CUDA;
    }
    return MD_OK;
}

md_status md_autotune(md_handle *h, int32_t trial_steps, int32_t *tile_max_out, void *stream)
{
    if (!h || trial_steps < 1) return fail(h, MD_ERR_ARG, "md_autotune: bad arguments");
    if (!h->state_set) return fail(h, MD_ERR_ARG, "md_autotune before md_set_state");
    cudaStream_t st = (cudaStream_t)stream;
    const long long n3 = 3 * h->N;
    // saved: x, v and the stored force in caller order, and the step counter
    double *save = dalloc<double>(h, (size_t)(3 * n3));
    if (!save) return fail(h, MD_ERR_CUDA, "cannot allocate");
    const bool had_F = h->F_valid;
    mdk::launch_get_state(h->b, save, save + n3, st);
    if (had_F) mdk::launch_force_by_id(h->b, save + 2 * n3, 0, st);
    if (!cuda_ok(h, cudaStreamSynchronize(st), "stream synchronize")) return MD_ERR_CUDA;
    Ctl c0;
    if (read_ctl(h, &c0) != MD_OK) return MD_ERR_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 0.f;
    int best = h->b.tile_max;
    md_status s = MD_OK;
    // the sweep of the paper's subnode count, from the largest task size: in
    // steps of 16 particles down to 64, every size tried (neighbouring sizes can
    // differ by less than a trial's noise, and a size that splits rows of cells
    // more evenly can win further down), then halving while it helps
    static const int kCands[] = {mdk::kTileMax, 112, 96, 80, 64, 32, 16, 8};
    for (int ci = 0; ci < (int)(sizeof(kCands) / sizeof(kCands[0])); ++ci) {
        const int cap = kCands[ci];
        if ((s = md_set_tile_size(h, cap, stream)) != MD_OK) break;
        if ((s = md_set_state(h, save, save + n3, st)) != MD_OK) break;
        if ((s = md_build_neighbors(h, stream)) != MD_OK) break;
        if ((s = md_step(h, 2, 0, nullptr, stream)) != MD_OK) break;
        cudaEventRecord(e0, st);
        if ((s = md_step(h, trial_steps, 0, nullptr, stream)) != MD_OK) break;
        cudaEventRecord(e1, st);
        if ((s = sync_and_check(h, st)) != MD_OK) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ci == 0 || ms < best_ms) { best_ms = ms; best = cap; }
        else if (cap <= 64) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s == MD_OK) s = md_set_tile_size(h, best, stream);
    if (s == MD_OK) s = md_set_state(h, save, save + n3, st);
    // the step counter (and with it the Langevin noise stream) carries on
    if (s == MD_OK && !cuda_ok(h, cudaMemcpyAsync(&h->b.ctl->step, &c0.step, sizeof(long long),
                                                  cudaMemcpyHostToDevice, st), "restore step"))
        s = MD_ERR_CUDA;
    if (s == MD_OK) s = md_build_neighbors(h, stream);
    // the stored force (with its Langevin terms) follows the re-sorted particles
    if (s == MD_OK && had_F) {
        mdk::launch_force_by_id(h->b, save + 2 * n3, 1, st);
        if (cuda_ok(h, cudaGetLastError(), "force restore")) h->F_valid = true;
        else s = MD_ERR_CUDA;
    }
    if (s == MD_OK) s = sync_and_check(h, st);
    cudaStreamSynchronize(st);
    for (auto it = h->allocs.begin(); it != h->allocs.end(); ++it)
        if (*it == save) { cudaFree(*it); h->allocs.erase(it); break; }
    if (tile_max_out) *tile_max_out = best;
    return s;
}

md_status md_set_timing(md_handle *h, int32_t enable)
{
    if (!h) return MD_ERR_ARG;
    if (!cuda_ok(h, cudaDeviceSynchronize(), "device synchronize")) return MD_ERR_CUDA;
    h->timing = enable != 0;
    h->ev_marks.clear();
    h->ev_used = 0;
    for (int k = 0; k < MD_NSECT; ++k) { h->sect_ms[k] = 0; h->sect_n[k] = 0; }
    return MD_OK;
}

md_status md_get_timing(md_handle *h, double *ms, int64_t *counts)
{
    if (!h) return MD_ERR_ARG;
    if (!cuda_ok(h, cudaDeviceSynchronize(), "device synchronize")) return MD_ERR_CUDA;
    resolve_timing(h);
    for (int k = 0; k < MD_NSECT; ++k) {
        if (ms) ms[k] = h->sect_ms[k];
        if (counts) counts[k] = h->sect_n[k];
    }
    return MD_OK;
}

const char *md_last_error(const md_handle *h) { return h ? h->err.c_str() : "null handle"; }

}  // extern "C"
