// Cell binning by counting sort, re-sort of the particle state into cell
// order, and Verlet-list build with a skin (arXiv:2109.10876 Sec. 2.1.2:
// particles are binned into cells of edge >= r_cut + r_skin, the pair search
// covers a particle's own cell and the 26 around it, and the list keeps every
// pair within r_cut + r_skin so it stays valid while particles move less than
// r_skin / 2).
//
// Every kernel here is launched on every step and returns at once unless
// Ctl::rebuild is set, so the decision to re-sort stays on the device.
#include "md_internal.cuh"

namespace mdk {

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ unsigned to_q(double y, double scale)
{
    // y in [0, L): y * 2^32 / L in [0, 2^32]; 2^32 wraps to 0 (periodic).
    return (unsigned)(fix_round(y, scale) & 0xffffffffLL);
}

__device__ __forceinline__ double wrap_box(double y, double L)
{
    if (y >= L || y < 0.0) {
        y = y - L * floor(y / L);
        if (y >= L) y = 0.0;
        if (y < 0.0) y = 0.0;
    }
    return y;
}

// Exact minimum-image squared distance in FP64 with a fixed rounding sequence:
// t = xi - xj; t -= L * rint(t / L) per axis; r2 = (dx^2 + dy^2) + dz^2.
// Used to settle pairs whose FP32 distance lies within rounding of a cutoff.
__device__ __noinline__ double r2_fp64(const double *x, long long S, long long i, long long j,
                                       const double *L)
{
    double d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double t = __dsub_rn(x[k * S + i], x[k * S + j]);
        double q = rint(__ddiv_rn(t, L[k]));
        double s = __dmul_rn(L[k], q);
        d[k] = __dsub_rn(t, s);
    }
    return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

__device__ __forceinline__ float r2_q(uint4 a, uint4 b, const float *qs)
{
    float dx = (float)(int)(a.x - b.x) * qs[0];
    float dy = (float)(int)(a.y - b.y) * qs[1];
    float dz = (float)(int)(a.z - b.z) * qs[2];
    return dx * dx + dy * dy + dz * dz;
}

__device__ __forceinline__ void cell_coords(uint4 p, const Replica &R, int &cx, int &cy, int &cz)
{
    cx = (int)(((unsigned long long)p.x * (unsigned)R.ncell[0]) >> 32);
    cy = (int)(((unsigned long long)p.y * (unsigned)R.ncell[1]) >> 32);
    cz = (int)(((unsigned long long)p.z * (unsigned)R.ncell[2]) >> 32);
}

// ---------------------------------------------------------------- state in/out
__global__ void k_reset_ctl(Ctl *ctl)
{
    ctl->cur = 0;
    ctl->rebuild = 1;
    ctl->disp2_bits = 0u;
    ctl->err = 0;
    ctl->done_force = ctl->done_list = ctl->done_kick = 0u;
    ctl->tile_next = 0u;
    ctl->max_occ = ctl->max_nn = 0;
    ctl->step = 0;
    ctl->rebuilds = 0;
    ctl->list_entries = 0;
    ctl->bad_site = 0;
    ctl->plant = 0;
    ctl->bad_index = 0;
    ctl->step0 = 0;
}

// Caller layout (3, N) -> slot layout; initial slot order = caller order.
__global__ void k_set_state(Bufs b, const double *xin, const double *vin)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.S) return;
    const Replica &R = b.rep[b.blk_rep[blockIdx.x]];
    long long local = s - R.slot_begin;
    double *x = b.x[0], *v = b.v[0];
    if (local < R.n) {
        long long id = R.id_begin + local;
        unsigned q[3];
        bool finite = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double y = xin[k * b.N + id];
            double w = vin[k * b.N + id];
            finite = finite && isfinite(y) && isfinite(w);
            y = isfinite(y) ? wrap_box(y, R.L[k]) : 0.0;
            x[k * b.S + s] = y;
            v[k * b.S + s] = w;
            q[k] = to_q(y, R.to_q[k]);
        }
        if (!finite) atomicOr(&b.ctl->err, kErrNonfinite);
        uint4 p = make_uint4(q[0], q[1], q[2], (unsigned)id);
        b.pos[0][s] = p;
        b.pos[1][s] = p;
        b.xref[s] = p;
        b.slot_of_id[id] = (int)s;
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) { x[k * b.S + s] = 0.0; v[k * b.S + s] = 0.0; }
        b.pos[0][s] = make_uint4(0u, 0u, 0u, 0xffffffffu);
        b.pos[1][s] = make_uint4(0u, 0u, 0u, 0xffffffffu);
        b.xref[s] = make_uint4(0u, 0u, 0u, 0xffffffffu);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) b.F[k * b.S + s] = 0.0;
    b.nn[s] = 0;
}

// Slot layout -> caller layout (3, N).
// Stored force between slot order and caller (id) order: dir 0 copies out,
// dir 1 copies in (after a re-sort, so that the stored force follows its
// particles).
__global__ void k_force_by_id(Bufs b, double *buf, int dir)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.S) return;
    int id = (int)b.pos[b.ctl->cur][s].w;
    if (id < 0) return;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (dir == 0) buf[k * b.N + id] = b.F[k * b.S + s];
        else b.F[k * b.S + s] = buf[k * b.N + id];
    }
}

__global__ void k_get_state(Bufs b, double *xout, double *vout)
{
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.S) return;
    int cur = b.ctl->cur;
    int id = (int)b.pos[cur][s].w;
    if (id < 0) return;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (xout) xout[k * b.N + id] = b.x[cur][k * b.S + s];
        if (vout) vout[k * b.N + id] = b.v[cur][k * b.S + s];
    }
}

__global__ void k_set_rebuild(Ctl *ctl) { ctl->rebuild = 1; }

// New positions (caller order) for the particles in their current slots: the
// slot order and the Verlet list stay, the fixed-point copies follow, and the
// largest displacement since the last list build is gathered as after a drift.
__global__ void __launch_bounds__(kBlock) k_reload(Bufs b, const double *xin)
{
    __shared__ float smax[kBlock / 32];
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float ratio = 0.0f;
    if (s < b.S) {
        const int cur = b.ctl->cur;
        const int id = (int)b.pos[cur][s].w;
        if (id >= 0) {
            const Replica &R = b.rep[b.blk_rep[blockIdx.x]];
            unsigned q[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double y = wrap_box(xin[k * b.N + id], R.L[k]);
                b.x[cur][k * b.S + s] = y;
                q[k] = to_q(y, R.to_q[k]);
            }
            const uint4 p = make_uint4(q[0], q[1], q[2], (unsigned)id);
            b.pos[cur][s] = p;
            const uint4 r = b.xref[s];
            const float dx = (float)(int)(p.x - r.x) * R.qs[0];
            const float dy = (float)(int)(p.y - r.y) * R.qs[1];
            const float dz = (float)(int)(p.z - r.z) * R.qs[2];
            ratio = (dx * dx + dy * dy + dz * dz) / R.disp2_thr;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ratio = fmaxf(ratio, __shfl_xor_sync(0xffffffffu, ratio, o));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = ratio;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kBlock / 32; ++w) ratio = fmaxf(ratio, smax[w]);
        if (ratio > 0.0f) atomicMax(&b.ctl->disp2_bits, __float_as_uint(ratio));
    }
}

// After k_reload: rebuild when some particle moved more than r_skin / 2.
__global__ void k_reload_decide(Ctl *ctl)
{
    const unsigned bits = atomicExch(&ctl->disp2_bits, 0u);
    ctl->rebuild = (__uint_as_float(bits) > 1.0f) ? 1 : 0;
}

__global__ void k_cond(Ctl *ctl, cudaGraphConditionalHandle handle, int what)
{
    const unsigned v = what == 0 ? (ctl->rebuild != 0 && ctl->err == 0) : (ctl->steps_left > 0 && ctl->err == 0);
    cudaGraphSetConditional(handle, v ? 1u : 0u);
}

__global__ void k_set_steps(Ctl *ctl, long long left)
{
    ctl->steps_left = left;
    ctl->rec = 0;
    ctl->step0 = ctl->step;
}

// The current positions in caller order into slot step - step0 of the
// position ring (a graph-launched md_step that records its trajectory).
__global__ void k_record_x(Bufs b)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.S) return;
    const int cur = b.ctl->cur;
    const int id = (int)b.pos[cur][s].w;
    if (id < 0) return;
    double *out = b.xring + 3 * b.N * (b.ctl->step - b.ctl->step0);
#pragma unroll
    for (int k = 0; k < 3; ++k) out[k * b.N + id] = b.x[cur][k * b.S + s];
}

// ---------------------------------------------------------------- counting sort
// a1: cell id of every particle and the cell histogram.  Slots are still in
// the previous build's cell order, so the lanes of a warp mostly share a few
// cells: one atomic per distinct cell of the warp (its lanes found by a match).
__global__ void k_bin(Bufs b)
{
    const unsigned full = 0xffffffffu;
    if (__shfl_sync(full, (int)(!b.ctl->rebuild || b.ctl->err), 0)) return;   // warp-uniform
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        b.ctl->max_nn = 0;
        b.ctl->list_entries = 0;
        b.ctl->max_occ = 0;
    }
    const int cur = b.ctl->cur;
    // a bounded grid strides over the blocks of kBlock slots (so that a launch
    // with no rebuild due costs little)
    for (int blk = blockIdx.x; blk < b.nblk; blk += gridDim.x) {
        const long long s = (long long)blk * blockDim.x + threadIdx.x;
        int c = -1;
        if (s < b.S) {
            const uint4 p = b.pos[cur][s];
            if ((int)p.w >= 0) {
                const Replica &R = b.rep[b.blk_rep[blk]];
                int cx, cy, cz;
                cell_coords(p, R, cx, cy, cz);
                c = R.cell_off + (cz * R.ncell[1] + cy) * R.ncell[0] + cx;
                if (md_ok(b.ctl, c >= R.cell_off && c < R.cell_off + R.ncells && c < b.C, kSiteBinCell, s))
                    b.cellid[s] = c;
                else
                    c = -1;
            }
        }
        const unsigned peers = __match_any_sync(full, c);
        if (c >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&b.cell_count[c], __popc(peers));
    }
}

constexpr int kScanThreads = 1024;

__device__ int block_excl_scan(int v, int *warp_sums, int &total)
{
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_sums[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int w = warp_sums[lane];
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        warp_sums[lane] = wi - w;   // exclusive prefix of warp totals
        if (lane == 31) warp_sums[32] = wi;
    }
    __syncthreads();
    int r = warp_sums[wid] + inc - v;
    total = warp_sums[32];
    __syncthreads();
    return r;
}

// The cell scan in three phases over blocks of kScanBlock cells: block sums
// (and the largest occupancy), an exclusive scan of the block sums, then each
// block's exclusive scan plus its offset.  Each replica's padding slots count
// after its last cell, so the result is the first slot of every cell.
__global__ void __launch_bounds__(kScanBlock) k_scan_sum(Bufs b)
{
    if (block_uniform(!b.ctl->rebuild || b.ctl->err)) return;
    __shared__ int warp_sums[33];
    const int c = blockIdx.x * kScanBlock + threadIdx.x;
    const int k = c < b.C ? b.cell_count[c] : 0;
    const int v = c < b.C ? k + b.cell_pad[c] : 0;
    int total;
    block_excl_scan(v, warp_sums, total);
    if (threadIdx.x == 0) b.scan_part[blockIdx.x] = total;
    int m = k;
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(&b.ctl->max_occ, m);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(Bufs b)
{
    if (block_uniform(!b.ctl->rebuild || b.ctl->err)) return;
    __shared__ int warp_sums[33];
    const int nb = (b.C + kScanBlock - 1) / kScanBlock;
    int carry = 0;
    for (int base = 0; base < nb; base += kScanThreads) {
        const int q = base + (int)threadIdx.x;
        const int v = q < nb ? b.scan_part[q] : 0;
        int total;
        const int e = block_excl_scan(v, warp_sums, total);
        if (q < nb) b.scan_part[q] = carry + e;
        carry += total;
    }
}

__global__ void __launch_bounds__(kScanBlock) k_scan_write(Bufs b)
{
    if (block_uniform(!b.ctl->rebuild || b.ctl->err)) return;
    __shared__ int warp_sums[33];
    const int c = blockIdx.x * kScanBlock + threadIdx.x;
    const int v = c < b.C ? b.cell_count[c] + b.cell_pad[c] : 0;
    int total;
    const int e = block_excl_scan(v, warp_sums, total) + b.scan_part[blockIdx.x];
    if (c < b.C) {
        b.cell_start[c] = e;
        b.cell_end[c] = e;   // cursor for the scatter
    }
}

// Scatter each particle's old slot into its cell's bucket (order within a
// cell is fixed afterwards by k_reorder): one atomic per distinct cell of the
// warp, its lanes taking consecutive places.
__global__ void k_scatter(Bufs b)
{
    const unsigned full = 0xffffffffu;
    if (__shfl_sync(full, (int)(!b.ctl->rebuild || b.ctl->err), 0)) return;   // warp-uniform
    const int lane = threadIdx.x & 31;
    const int cur = b.ctl->cur;
    for (int blk = blockIdx.x; blk < b.nblk; blk += gridDim.x) {   // bounded grid, as k_bin
        const long long s = (long long)blk * blockDim.x + threadIdx.x;
        int c = -1;
        if (s < b.S && (int)b.pos[cur][s].w >= 0) c = b.cellid[s];
        const unsigned peers = __match_any_sync(full, c);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (c >= 0 && lane == leader) base = atomicAdd(&b.cell_end[c], __popc(peers));
        base = __shfl_sync(full, base, leader);
        if (c >= 0) {
            const int dst = base + __popc(peers & ((1u << lane) - 1u));
            const int lim = c + 1 < b.C ? b.cell_start[c + 1] : (int)b.S;
            if (md_ok(b.ctl, dst >= b.cell_start[c] && dst < lim, kSiteScatter, dst)) b.bucket[dst] = (int)s;
        }
    }
}

// One warp per cell: order the cell's members by (fixed-point x, particle
// id), a function of the positions alone, so that every row of cells is
// sorted along x; then gather x, v, pos from buffer cur into buffer cur ^ 1
// at the new slots.  Ranks come from warp shuffles for cells of up to 32.
__device__ __forceinline__ unsigned long long order_key(uint4 p)
{
    return ((unsigned long long)p.x << 32) | (unsigned)p.w;
}

__device__ __forceinline__ void reorder_move(const Bufs &b, int cur, int nxt, int c, int s, int dst, uint4 p)
{
    if (!md_ok(b.ctl, (int)p.w >= 0 && (long long)p.w < b.N && dst >= 0 && dst < b.S, kSiteReorder, dst)) return;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        b.x[nxt][k * b.S + dst] = b.x[cur][k * b.S + s];
        b.v[nxt][k * b.S + dst] = b.v[cur][k * b.S + s];
    }
    b.pos[nxt][dst] = p;
    b.xref[dst] = p;
    b.slot_of_id[(int)p.w] = dst;
    b.cellid[dst] = c;
}

// One cell (first slot start, n members) by a whole warp: ranks by shuffles
// for up to 32 members, by a loop over the members beyond.
__device__ __forceinline__ void reorder_cell_warp(const Bufs &b, int cur, int nxt, int c, int start, int n,
                                                  int lane)
{
    const uint4 *pin = b.pos[cur];
    if (n <= 32) {
        const bool act = lane < n;
        int s = act ? b.bucket[start + lane] : 0;
        if (act && !md_ok(b.ctl, s >= 0 && s < b.S, kSiteReorder, s)) s = 0;
        const uint4 p = act ? pin[s] : make_uint4(0u, 0u, 0u, 0u);
        const unsigned long long key = act ? order_key(p) : ~0ULL;
        int rank = 0;
        for (int q = 0; q < n; ++q) rank += (__shfl_sync(0xffffffffu, key, q) < key);
        if (act) reorder_move(b, cur, nxt, c, s, start + rank, p);
        return;
    }
    for (int m = lane; m < n; m += 32) {
        int s = b.bucket[start + m];
        if (!md_ok(b.ctl, s >= 0 && s < b.S, kSiteReorder, s)) s = 0;
        uint4 p = pin[s];
        const unsigned long long key = order_key(p);
        int rank = 0;
        for (int q = 0; q < n; ++q) {
            int sq = b.bucket[start + q];
            if (!md_ok(b.ctl, sq >= 0 && sq < b.S, kSiteReorder, sq)) sq = 0;
            rank += (order_key(pin[sq]) < key);
        }
        reorder_move(b, cur, nxt, c, s, start + rank, p);
    }
}

// A warp takes four cells at a time: a cell of at most 8 members is ordered
// by its own 8 lanes (ranks by shuffles within the group; keys are unique and
// idle lanes hold the largest), and the group's larger cells go to the whole
// warp one after another.  Sparse systems (a melt's three particles per cell,
// a vapour's fraction of one) then keep most lanes busy.
__global__ void k_reorder(Bufs b)
{
    if (!b.ctl->rebuild || b.ctl->err) return;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, g = lane >> 3, gl = lane & 7;
    const int cur = b.ctl->cur, nxt = cur ^ 1;
    const uint4 *pin = b.pos[cur];
    // a bounded grid of warps strides over groups of four cells
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long c0 = 4 * (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5); c0 < b.C; c0 += 4 * nw) {
        const long long cl = c0 + g;
        int start = 0, n = 0;
        if (cl < b.C) {
            start = b.cell_start[cl];
            n = b.cell_end[cl] - start;
            if (gl == 0) b.cell_count[cl] = 0;   // histogram is clean for the next build
        }
        const bool small = cl < b.C && n <= 8;
        if (__any_sync(full, small)) {   // warp-uniform: a dense system skips this part
            const bool act = small && gl < n;
            int s = act ? b.bucket[start + gl] : 0;
            if (act && !md_ok(b.ctl, s >= 0 && s < b.S, kSiteReorder, s)) s = 0;
            const uint4 p = act ? pin[s] : make_uint4(0u, 0u, 0u, 0u);
            const unsigned long long key = act ? order_key(p) : ~0ULL;
            int rank = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) rank += (__shfl_sync(full, key, (lane & ~7) | q) < key);
            if (act) reorder_move(b, cur, nxt, (int)cl, s, start + rank, p);
        }
        unsigned big = __ballot_sync(full, gl == 0 && cl < b.C && !small);
        while (big) {
            const int lead = __ffs(big) - 1;
            big &= big - 1;
            const int bs = __shfl_sync(full, start, lead), bn = __shfl_sync(full, n, lead);
            reorder_cell_warp(b, cur, nxt, (int)(c0 + (lead >> 3)), bs, bn, lane);
        }
    }
}

// Slots of the bond partners and of the members of the angle triples, per
// entry of the (particle-id ordered) bond and triple tables.  Slots change
// only when the particles are re-sorted, so this runs once per rebuild and
// the force kernel reads one entry per bond or triple instead of mapping
// particle ids to slots every step.
__global__ void k_topology_slots(Bufs b)
{
    if (!b.ctl->rebuild || b.ctl->err) return;
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    auto id_ok = [&](int id) { return md_ok(b.ctl, id >= 0 && id < b.N, kSiteTopology, id); };
    if (q < b.n_bond_ent) {
        const int id = b.bond_partner[q];
        b.bond_pslot[q] = id_ok(id) ? b.slot_of_id[id] : 0;
    }
    if (q < b.n_ang_ent) {
        const int4 e = b.ang_ent[q];
        const bool ok = id_ok(e.x) & id_ok(e.y) & id_ok(e.z);
        b.ang_slot[q] = ok ? make_int4(b.slot_of_id[e.x], b.slot_of_id[e.y], b.slot_of_id[e.z], e.w)
                           : make_int4(0, 0, 0, e.w);
    }
}

// ---------------------------------------------------------------- tiles
// Rows of all replica grids are numbered replica by replica, cz-major; a warp
// walks one row.  Lanes first sum, for every column x of the row, the
// particles in that column of the (up to) 3 x 3 neighbouring rows; lane 0
// then cuts the row greedily into tiles of at most kTileMax particles whose
// halo (columns x0 - 1 .. x1 of those rows) holds at most hcap particles.
constexpr int kTileWarps = 4;
constexpr int kRowMax = 1024;   // columns held in shared memory per warp

__device__ __forceinline__ int cell_n(const Bufs &b, int c) { return b.cell_end[c] - b.cell_start[c]; }

// Walk one row; writes tiles to out (if non-null) and returns their count.
__device__ int walk_row(const Bufs &b, int g, Tile *out, int *colsum, int *own)
{
    const int r = b.row_rep[g];
    const Replica &R = b.rep[r];
    const int nx = R.ncell[0], ny = R.ncell[1], nz = R.ncell[2];
    const int lr = g - R.row_off;                // row index within the replica
    const int cy = lr % ny, cz = lr / ny;
    int ly, cntY, lz, cntZ;
    axis_offsets(ny, ly, cntY);
    axis_offsets(nz, lz, cntZ);
    const int lane = threadIdx.x & 31;
    const bool in_smem = nx <= kRowMax;
    if (in_smem) {
        for (int x = lane; x < nx; x += 32) {
            int sum = 0;
            for (int oz = 0; oz < cntZ; ++oz)
                for (int oy = 0; oy < cntY; ++oy) {
                    int zz = wrapi(cz + lz + oz, nz), yy = wrapi(cy + ly + oy, ny);
                    sum += cell_n(b, R.cell_off + (zz * ny + yy) * nx + x);
                }
            colsum[x] = sum;
            own[x] = cell_n(b, R.cell_off + (cz * ny + cy) * nx + x);
        }
    }
    __syncwarp();
    int nt = 0;
    if (in_smem) {
        // inclusive prefix sums of the column halo counts and of the row's own
        // counts, in place: the greedy cut below then needs no serial walk
        const unsigned full = 0xffffffffu;
        int carry_c = 0, carry_o = 0;
        for (int base = 0; base < nx; base += 32) {
            const int x = base + lane;
            int vc = x < nx ? colsum[x] : 0, vo = x < nx ? own[x] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int tc = __shfl_up_sync(full, vc, o), to = __shfl_up_sync(full, vo, o);
                if (lane >= o) { vc += tc; vo += to; }
            }
            vc += carry_c;
            vo += carry_o;
            if (x < nx) { colsum[x] = vc; own[x] = vo; }
            carry_c = __shfl_sync(full, vc, 31);
            carry_o = __shfl_sync(full, vo, 31);
        }
        __syncwarp();
        if (lane == 0) {
            // tile [x0, x1): P = its own particles, H = the halo columns x0 - 1 .. x1
            // (wrapped), or the whole row's halo where that many columns reach round
            // it.  Both only grow with x1, so the greedy end of a tile (the largest
            // x1 that keeps P <= tile_max and H <= hcap, and at least one cell) is
            // found by a binary search.
            const int *PC = colsum, *PO = own;
            const int total = PC[nx - 1];
            auto pc_at = [&](int x) -> int { return x < 0 ? 0 : PC[x]; };
            auto halo = [&](int x0, int x1) -> int {
                if (x1 - x0 + 2 >= nx) return total;
                int a = x0 - 1, e = x1, h = 0;
                if (a < 0) { h += PC[nx - 1] - PC[nx - 2]; a = 0; }
                if (e >= nx) { h += PC[0]; e = nx - 1; }
                return h + PC[e] - pc_at(a - 1);
            };
            auto fits = [&](int x0, int x1) -> bool {
                return PO[x1 - 1] - (x0 > 0 ? PO[x0 - 1] : 0) <= b.tile_max && halo(x0, x1) <= b.hcap;
            };
            int x0 = 0;
            while (x0 < nx) {
                int x1 = x0 + 1;
                if (fits(x0, x1)) {
                    int lo = x1, hi = nx;
                    while (lo < hi) {
                        const int m = (lo + hi + 1) >> 1;
                        if (fits(x0, m)) lo = m; else hi = m - 1;
                    }
                    x1 = lo;
                }
                if (out && md_ok(b.ctl, (out - b.tiles) + nt < b.C, kSiteTileWrite, (out - b.tiles) + nt)) {
                    const int base = R.cell_off + (cz * ny + cy) * nx;
                    Tile t;
                    t.rep = r; t.cy = cy; t.cz = cz; t.x0 = x0; t.x1 = x1;
                    t.s0 = b.cell_start[base + x0];
                    t.s1 = b.cell_end[base + x1 - 1];
                    t.hsize = halo(x0, x1);
                    t.kmax = 0;
                    out[nt] = t;
                }
                ++nt;
                x0 = x1;
            }
        }
    } else if (lane == 0) {
        // a row wider than the shared arrays: the serial walk over its columns
        auto col = [&](int x) -> int {
            if (in_smem) return colsum[x];
            int sum = 0;
            for (int oz = 0; oz < cntZ; ++oz)
                for (int oy = 0; oy < cntY; ++oy) {
                    int zz = wrapi(cz + lz + oz, nz), yy = wrapi(cy + ly + oy, ny);
                    sum += cell_n(b, R.cell_off + (zz * ny + yy) * nx + x);
                }
            return sum;
        };
        auto mine = [&](int x) -> int { return in_smem ? own[x] : cell_n(b, R.cell_off + (cz * ny + cy) * nx + x); };
        int total = 0;
        for (int x = 0; x < nx; ++x) total += col(x);
        int x0 = 0;
        while (x0 < nx) {
            // halo of [x0, x0 + 1): columns x0 - 1, x0, x0 + 1 (or the whole row)
            int x1 = x0 + 1;
            int P = mine(x0);
            int H = (3 >= nx) ? total : col(wrapi(x0 - 1, nx)) + col(x0) + col(wrapi(x0 + 1, nx));
            while (x1 < nx) {
                const int c = mine(x1);
                const int Hn = (x1 + 1 - x0 + 2 >= nx) ? total : H + col(wrapi(x1 + 1, nx));
                if (P + c > b.tile_max || Hn > b.hcap) break;
                P += c;
                H = Hn;
                ++x1;
            }
            if (out && md_ok(b.ctl, (out - b.tiles) + nt < b.C, kSiteTileWrite, (out - b.tiles) + nt)) {
                const int base = R.cell_off + (cz * ny + cy) * nx;
                Tile t;
                t.rep = r; t.cy = cy; t.cz = cz; t.x0 = x0; t.x1 = x1;
                t.s0 = b.cell_start[base + x0];
                t.s1 = b.cell_end[base + x1 - 1];
                t.hsize = H;
                t.kmax = 0;
                out[nt] = t;
            }
            ++nt;
            x0 = x1;
        }
    }
    __syncwarp();
    return nt;
}

__global__ void __launch_bounds__(32 * kTileWarps) k_tile_count(Bufs b)
{
    if (!b.ctl->rebuild || b.ctl->err) return;
    __shared__ int colsum[kTileWarps][kRowMax], own[kTileWarps][kRowMax];
    const int w = threadIdx.x >> 5;
    const int g = blockIdx.x * kTileWarps + w;
    if (g >= b.nrows) return;
    int nt = walk_row(b, g, nullptr, colsum[w], own[w]);
    if ((threadIdx.x & 31) == 0) b.row_tiles[g] = nt;
}

// Exclusive scan of tiles per row (one block); first tile of every replica.
__global__ void __launch_bounds__(kScanThreads) k_tile_scan(Bufs b)
{
    if (block_uniform(!b.ctl->rebuild || b.ctl->err)) return;
    __shared__ int warp_sums[33];
    const int n = b.nrows;
    const int chunk = (n + kScanThreads - 1) / kScanThreads;
    const int lo = min(n, (int)threadIdx.x * chunk), hi = min(n, lo + chunk);
    int sum = 0;
    for (int g = lo; g < hi; ++g) sum += b.row_tiles[g];
    int total;
    int base = block_excl_scan(sum, warp_sums, total);
    for (int g = lo; g < hi; ++g) {
        const int t = b.row_tiles[g];
        b.row_tiles[g] = base;
        if (g == 0 || b.row_rep[g - 1] != b.row_rep[g]) b.rep_tile[b.row_rep[g]] = base;
        base += t;
    }
    if (threadIdx.x == 0) {
        b.row_tiles[n] = total;
        b.rep_tile[b.nrep] = total;
        for (int r = b.nrep - 1; r >= 0; --r)   // replicas without rows (none in practice)
            if (b.rep[r].ncells == 0) b.rep_tile[r] = b.rep_tile[r + 1];
        b.ctl->ntiles = total;
        b.ctl->max_halo = 0;
    }
}

__global__ void __launch_bounds__(32 * kTileWarps) k_tile_write(Bufs b)
{
    if (!b.ctl->rebuild || b.ctl->err) return;
    __shared__ int colsum[kTileWarps][kRowMax], own[kTileWarps][kRowMax];
    const int w = threadIdx.x >> 5;
    const int g = blockIdx.x * kTileWarps + w;
    if (g >= b.nrows) return;
    walk_row(b, g, b.tiles + b.row_tiles[g], colsum[w], own[w]);
}

// Halo pieces of every tile, computed once per build: a warp per tile, lane
// r computing the slot ranges of halo row r; a warp prefix sum places them.
__global__ void __launch_bounds__(32 * kTileWarps) k_tile_pieces(Bufs b)
{
    if (!b.ctl->rebuild || b.ctl->err) return;
    const int lane = threadIdx.x & 31;
    const int nt = b.ctl->ntiles;
    // a bounded grid walks the tiles (their count is known on the device only)
    for (int t = blockIdx.x * kTileWarps + (threadIdx.x >> 5); t < nt; t += gridDim.x * kTileWarps) {
        const Tile tl = b.tiles[t];
        const Replica &R = b.rep[tl.rep];
        const int nx = R.ncell[0], ny = R.ncell[1], nz = R.ncell[2];
        int ly, cntY, lz, cntZ;
        axis_offsets(ny, ly, cntY);
        axis_offsets(nz, lz, cntZ);
        const int nrow = cntY * cntZ;
        int npc = 0, cnt[2] = {0, 0}, ra[2] = {0, 0}, rb[2] = {0, 0}, s0[2] = {0, 0};
        if (lane < nrow) {
            const int oz = lane / cntY, oy = lane - oz * cntY;
            const int zz = wrapi(tl.cz + lz + oz, nz), yy = wrapi(tl.cy + ly + oy, ny);
            const int base = R.cell_off + (zz * ny + yy) * nx;
            const int x0 = tl.x0, x1 = tl.x1;
            if (x1 - x0 + 2 >= nx) { ra[0] = 0; rb[0] = nx; npc = 1; }
            else if (x0 == 0) { ra[0] = nx - 1; rb[0] = nx; ra[1] = 0; rb[1] = x1 + 1; npc = 2; }
            else if (x1 == nx) { ra[0] = x0 - 1; rb[0] = nx; ra[1] = 0; rb[1] = 1; npc = 2; }
            else { ra[0] = x0 - 1; rb[0] = x1 + 1; npc = 1; }
            for (int q = 0; q < npc; ++q) {
                s0[q] = b.cell_start[base + ra[q]];
                cnt[q] = b.cell_end[base + rb[q] - 1] - s0[q];
            }
        }
        // exclusive prefix over lanes of pieces and halo sizes
        int pinc = npc, hinc = cnt[0] + cnt[1];
        for (int o = 1; o < 32; o <<= 1) {
            const int a = __shfl_up_sync(0xffffffffu, pinc, o), c = __shfl_up_sync(0xffffffffu, hinc, o);
            if (lane >= o) { pinc += a; hinc += c; }
        }
        const int pbase = pinc - npc, hbase = hinc - (cnt[0] + cnt[1]);
        Piece *out = b.pieces + (size_t)t * (kMaxPieces + 1);
        int h = hbase;
        for (int q = 0; q < npc; ++q) {
            Piece pq;
            pq.row = lane; pq.xa = ra[q]; pq.xb = rb[q]; pq.slot0 = s0[q]; pq.hoff = h; pq.n = cnt[q];
            // a piece's slots lie within the slots (its bulk copy reads them)
            if (md_ok(b.ctl, pbase + q < kMaxPieces && s0[q] >= 0 && cnt[q] >= 0 && s0[q] + cnt[q] <= b.S,
                      kSitePieces, (long long)t * (kMaxPieces + 1) + pbase + q))
                out[pbase + q] = pq;
            h += cnt[q];
        }
        const int np = __shfl_sync(0xffffffffu, pinc, 31), H = __shfl_sync(0xffffffffu, hinc, 31);
        if (lane == 0 && md_ok(b.ctl, np <= kMaxPieces, kSitePieces, (long long)t * (kMaxPieces + 1) + np)) {
            Piece last;
            last.row = nrow; last.xa = last.xb = 0; last.slot0 = 0; last.hoff = H; last.n = 0;
            out[np] = last;
            b.tile_np[t] = np;
            atomicMax(&b.ctl->max_halo, H);
        }
    }
}

// ---------------------------------------------------------------- list build
// a2: Verlet list of every pair within r_cut + r_skin.  A persistent block
// takes tiles from a work counter and stages the tile's halo positions in
// shared memory.  Each warp takes one cell of the tile at a time, its lanes
// the cell's particles; the lanes walk the neighbouring cells (found in the
// halo) in step, reading each candidate once for the whole warp, and keep the
// halo index of every partner.  The FP32 distance decides all pairs except
// those within its rounding of the list radius, which are settled in FP64
// from the master positions (same formula as the FP64 reference), so the list
// is exactly the FP64 pair set.  Lists are staged in shared memory and leave
// as contiguous rows of the tile layout.

__host__ __device__ inline size_t list_smem_bytes(int hcap)
{
    return (size_t)hcap * sizeof(uint4) + (size_t)(kListStage * kTileMax + 32) * sizeof(unsigned short);
}

// Lists of the particles of one tile.  A warp takes 32 consecutive particles
// of the tile, one per lane (they span one to a few cells of the tile's row),
// and walks the union of their stencils -- on each of the 3 x 3 halo rows,
// the cells from one left of the first particle's cell to one right of the
// last one's -- with every lane reading the same candidate at a time.  A
// candidate outside a lane's own 27 cells is at least a cell edge (>= r_cut +
// r_skin) away and fails the distance test, so each list is exactly the pair
// set, ordered by halo row and slot.  Distances in fixed-point units of the
// x axis (see Replica).
// Halo entries of the list walk, in one of two forms.
// Relative (REL): FP32 coordinates relative to the tile centre in x-axis
// fixed-point units, w = the halo index.  With at least 3 cells in y and z
// and a tile at least 3 cells narrower than its row, no halo coordinate wraps
// around the centre (offsets stay below L / 2) and every tile-halo pair spans
// less than L - r_list along each axis, so the difference of two entries is
// the minimum image wherever that can be below r_list.  It saves the
// per-candidate integer-to-float conversions.
// Absolute: the fixed-point positions; the int32 difference is the minimum
// image in every case.
template <bool REL> struct Cand;
template <> struct Cand<true> {
    using T = float4;
    __device__ static float sep2(const float4 &p, const float4 &q, float, float)
    {
        const float d0 = p.x - q.x, d1 = p.y - q.y, d2 = p.z - q.z;
        return d0 * d0 + d1 * d1 + d2 * d2;
    }
    __device__ static int index(const float4 &q, int) { return __float_as_int(q.w); }
    // two candidates at once with packed FP32 instructions (the same
    // operations per lane; the negation is exact)
    __device__ static float2 sep2x2(const float4 &p, const float4 &q0, const float4 &q1, float, float)
    {
        const float2 d0 = __fadd2_rn(make_float2(p.x, p.x), make_float2(-q0.x, -q1.x));
        const float2 d1 = __fadd2_rn(make_float2(p.y, p.y), make_float2(-q0.y, -q1.y));
        const float2 d2 = __fadd2_rn(make_float2(p.z, p.z), make_float2(-q0.z, -q1.z));
        return __ffma2_rn(d2, d2, __ffma2_rn(d1, d1, __fmul2_rn(d0, d0)));
    }
};
template <> struct Cand<false> {
    using T = uint4;
    __device__ static float sep2(const uint4 &p, const uint4 &q, float ry, float rz)
    {
        const float d0 = (float)(int)(p.x - q.x);
        const float d1 = (float)(int)(p.y - q.y) * ry;
        const float d2 = (float)(int)(p.z - q.z) * rz;
        return d0 * d0 + d1 * d1 + d2 * d2;
    }
    __device__ static int index(const uint4 &, int h) { return h; }
    __device__ static float2 sep2x2(const uint4 &p, const uint4 &q0, const uint4 &q1, float ry, float rz)
    {
        return make_float2(sep2(p, q0, ry, rz), sep2(p, q1, ry, rz));
    }
};

// Halo range `lane` (< 2 nrow) of the union of the stencils of particles
// [g0, g1] of the tile (cells [xa - 1, xb + 1] on each of the nrow halo rows,
// split at the periodic boundary), trimmed for REL to the x-window of the
// first and last of those particles.  Returns (h0, h1, j0): halo indices
// [h0, h1) with first slot j0; empty for other lanes or an empty group.
template <bool REL>
__device__ __forceinline__ void union_range(const Bufs &b, const Replica &R, const Tile &tl, const Piece *pc, int np,
                                            const typename Cand<REL>::T *halo, int hfirst, int g0, int g1, int lane,
                                            int &rh0, int &rh1, int &rj0, int &err)
{
    const int nx = R.ncell[0], ny = R.ncell[1], nz = R.ncell[2];
    int ly, cntY, lz, cntZ;
    axis_offsets(ny, ly, cntY);
    axis_offsets(nz, lz, cntZ);
    const int nrow = cntY * cntZ;
    rh0 = rh1 = rj0 = 0;
    if (g0 > g1 || lane >= nrow * 2) return;
    const int xa = (b.cellid[tl.s0 + g0] - R.cell_off) % nx;
    const int xb = (b.cellid[tl.s0 + g1] - R.cell_off) % nx;
    const bool whole = xb - xa + 3 >= nx;
    const int row = lane >> 1, part = lane & 1;
    const int oz = row / cntY, oy = row - oz * cntY;
    const int zz = wrapi(tl.cz + lz + oz, nz), yy = wrapi(tl.cy + ly + oy, ny);
    const int base = R.cell_off + (zz * ny + yy) * nx;
    int ca = -1, cb = -1;     // cells [ca, cb) of this part
    if (whole) { if (part == 0) { ca = 0; cb = nx; } }
    else {
        const int a = xa - 1, e = xb + 2;    // [a, e) before wrapping
        if (a < 0) { if (part == 0) { ca = a + nx; cb = nx; } else { ca = 0; cb = e; } }
        else if (e > nx) { if (part == 0) { ca = a; cb = nx; } else { ca = 0; cb = e - nx; } }
        else if (part == 0) { ca = a; cb = e; }
    }
    if (!(ca >= 0 && cb > ca)) return;
    int qq = 0;
    while (qq + 1 < np && !(pc[qq].row == row && pc[qq].xa <= ca && ca < pc[qq].xb)) ++qq;
    const int j0 = b.cell_start[base + ca], j1 = b.cell_end[base + cb - 1];
    rh0 = pc[qq].hoff + (j0 - pc[qq].slot0);
    rh1 = rh0 + (j1 - j0);
    rj0 = j0;
    if (rh0 < pc[qq].hoff || rh1 > pc[qq].hoff + pc[qq].n) { err |= kErrList; rh1 = rh0; return; }
    if (!md_ok(b.ctl, rh0 >= 0 && rh1 <= pc[np].hoff, kSiteListRange, rh1)) { rh0 = rh1 = 0; return; }
    if constexpr (REL) {
        // Rows are sorted along x (cells in order, members by x), and so are
        // the group's own particles: candidates farther along x than the
        // window from the first and last of them are out of reach of all.
        const float xlo = halo[hfirst + g0].x - R.rl_win_u;
        const float xhi = halo[hfirst + g1].x + R.rl_win_u;
        int a = rh0, e = rh1;
        while (a < e) {
            const int m = (a + e) >> 1;
            if (halo[m].x < xlo) a = m + 1; else e = m;
        }
        int a2 = a;
        e = rh1;
        while (a2 < e) {
            const int m = (a2 + e) >> 1;
            if (halo[m].x <= xhi) a2 = m + 1; else e = m;
        }
        rj0 += a - rh0;
        rh0 = a;
        rh1 = a2;
    }
}

// The tile-relative form of union_range, for both groups of a warp at once:
// lane q takes halo piece q (a run of consecutive cells of one halo row, sorted
// along x) and keeps, for each group, the entries whose x lies in the group's
// window [x of its first particle - w, x of its last + w].  The window lies
// within the cells one left of the group's first cell to one right of its last
// (the cell edge is at least the list radius), so these are the candidates of
// the cell ranges trimmed to the window, found without the cells' slot bounds
// from global memory.  The four bounds (two per group) are counts of entries
// below a value, taken in lockstep by power-of-two steps (a fixed number of
// steps for the piece, no branches), so their shared-memory reads overlap.
__device__ __forceinline__ void union_ranges_rel(const Bufs &b, const Replica &R, const Piece *pc, int np,
                                                 const float4 *halo, int hfirst, int c0, int Pt, int lane,
                                                 int (*rng)[kMaxPieces][3])
{
    int r[2][3] = {{0, 0, 0}, {0, 0, 0}};
    if (lane < np && pc[lane].n > 0) {
        const Piece q = pc[lane];
        const float w = R.rl_win_u;
        const int g0a = c0, g1a = min(c0 + 15, Pt - 1), g0b = c0 + 16, g1b = min(c0 + 31, Pt - 1);
        const bool vb = g0b <= g1b;
        const float loA = halo[hfirst + g0a].x - w, hiA = halo[hfirst + g1a].x + w;
        const float loB = vb ? halo[hfirst + g0b].x - w : loA, hiB = vb ? halo[hfirst + g1b].x + w : hiA;
        const float4 *x = halo + q.hoff;
        const int n = q.n;
        int cA0 = 0, cA1 = 0, cB0 = 0, cB1 = 0;   // entries with x < loA, x <= hiA, x < loB, x <= hiB
        for (int step = 1 << (31 - __clz(n)); step > 0; step >>= 1) {
            if (cA0 + step <= n && x[cA0 + step - 1].x < loA) cA0 += step;
            if (cA1 + step <= n && x[cA1 + step - 1].x <= hiA) cA1 += step;
            if (cB0 + step <= n && x[cB0 + step - 1].x < loB) cB0 += step;
            if (cB1 + step <= n && x[cB1 + step - 1].x <= hiB) cB1 += step;
        }
        if (md_ok(b.ctl, cA0 <= cA1 && cB0 <= cB1 && q.hoff + n <= pc[np].hoff, kSiteListRange, q.hoff + n)) {
            r[0][0] = q.hoff + cA0; r[0][1] = q.hoff + cA1; r[0][2] = q.slot0 + cA0;
            if (vb) { r[1][0] = q.hoff + cB0; r[1][1] = q.hoff + cB1; r[1][2] = q.slot0 + cB0; }
        }
    }
    if (lane < np) {
#pragma unroll
        for (int k = 0; k < 3; ++k) { rng[0][lane][k] = r[0][k]; rng[1][lane][k] = r[1][k]; }
    }
}

// Verlet lists of one tile (Sec. 2.1.2).  Each half-warp takes 16
// consecutive particles and walks the union of their 27-cell stencils,
// candidate by candidate (a shared-memory broadcast per half), keeping j when
// |d_ij| < r_cut + r_skin.  The ranges of both unions sit in the warp's table
// `rng` ([half][range][h0, h1, j0]), so no loop below needs the other lanes:
// the two halves run their own ranges side by side.  The walk keeps every
// candidate whose FP32 r^2 is below the upper edge of the rounding band of
// the list radius; a lane that kept one inside the band (rare) afterwards
// drops those whose FP64 distance from the master positions is not below the
// radius.  Appends are branch-free: every candidate is written at the lane's
// next free row and the row pointer advances only on a hit.  The shared stage
// has the final [row][particle] layout of the tile's list block; a list that
// outgrows it is walked again straight into global memory (rare).
// HALF: the half list of Newton's third law (Sec. 2.1.2), each pair once, in
// the list of the particle with the lower slot: candidate h of range r has
// slot j0 + (h - h0), so it is kept only when h > i - j0 + h0.  Every pair of
// the full list survives in exactly one of its two lists (slots are unique).
template <bool REL, bool HALF>
__device__ __forceinline__ void cells_of_tile(const Bufs &b, const Replica &R, const Tile &tl, const Piece *pc, int np,
                                              const typename Cand<REL>::T *halo, unsigned short *lst, const double *X,
                                              int hfirst, int (*rng)[kMaxPieces][3], int *s_kmax, int &mx,
                                              long long &sm, int &err)
{
    using C = Cand<REL>;
    using T = typename C::T;
    const float ry = R.ry, rz = R.rz;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int half = lane >> 4;
    int ly, cntY, lz, cntZ;
    axis_offsets(R.ncell[1], ly, cntY);
    axis_offsets(R.ncell[2], lz, cntZ);
    // ranges per group: one per halo piece in the tile-relative form, else one
    // per (halo row, side of the periodic boundary)
    const int nrng = REL ? np : 2 * cntY * cntZ;
    const float lo = R.rl2_lo_u, hi = R.rl2_hi_u;
    const int Pt = tl.s1 - tl.s0;
    // stage rows of this tile (0: no stage, every list goes to global memory)
    const int cap = Pt <= kTileMax ? min((kListStage * kTileMax) / max(Pt, 1), b.K) : 0;
    unsigned short *dummy = lst + kListStage * kTileMax;     // one slot per lane
    // the tile's own particles are halo entries [hfirst, hfirst + Pt) (same
    // decision in every thread)
    if (!md_ok(b.ctl, hfirst >= 0 && hfirst + Pt <= pc[np].hoff, kSiteListSelf, hfirst)) return;
    for (int c0 = warp * 32; c0 < Pt; c0 += nwarp * 32) {
        const int pp = c0 + lane;
        const bool valid = pp < Pt;
        const int i = tl.s0 + (valid ? pp : c0);
        if constexpr (REL) {
            union_ranges_rel(b, R, pc, np, halo, hfirst, c0, Pt, lane, rng);
        } else {
            int h0, h1, j0;
            union_range<REL>(b, R, tl, pc, np, halo, hfirst, c0, min(c0 + 15, Pt - 1), lane, h0, h1, j0, err);
            if (lane < nrng) { rng[0][lane][0] = h0; rng[0][lane][1] = h1; rng[0][lane][2] = j0; }
            union_range<REL>(b, R, tl, pc, np, halo, hfirst, c0 + 16, min(c0 + 31, Pt - 1), lane, h0, h1, j0, err);
            if (lane < nrng) { rng[1][lane][0] = h0; rng[1][lane][1] = h1; rng[1][lane][2] = j0; }
        }
        __syncwarp();
        const int self = valid ? hfirst + pp : -1;
        const T p = halo[hfirst + (valid ? pp : c0)];
        // this lane's stage column (row stride Pt); lanes without one write a
        // private dummy slot (stride 0)
        const bool own = valid && cap > 0;
        unsigned short *col = own ? lst + pp : dummy + lane;
        const int stride = own ? Pt : 0;
        int cnt = 0;
        bool tie = false;    // a kept candidate lies within rounding of the list radius
        for (int r = 0; r < nrng; ++r) {
            const int h1 = rng[half][r][1];
            int h = rng[half][r][0];
            const int thr = HALF ? i - rng[half][r][2] + h : 0;   // HALF: keep halo indices above thr
            for (; h + 4 <= h1; h += 4) {
                T pj[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) pj[u] = halo[h + u];
                float r2v[4];
#pragma unroll
                for (int u = 0; u < 4; u += 2) {
                    const float2 r = C::sep2x2(p, pj[u], pj[u + 1], ry, rz);
                    r2v[u] = r.x;
                    r2v[u + 1] = r.y;
                }
                // four free rows from here while cnt <= cap - 4 (else re-walked below)
                unsigned short *q = col + max(min(cnt, cap - 4), 0) * stride;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float r2 = r2v[u];
                    const int hj = C::index(pj[u], h + u);
                    const bool flt = HALF ? hj > thr : hj != self;
                    const bool in = (r2 < hi) & flt;
                    tie |= in & !(r2 < lo);
                    *q = (unsigned short)hj;
                    q += in ? stride : 0;
                    cnt += in;
                }
            }
            for (; h < h1; ++h) {
                const float r2 = C::sep2(p, halo[h], ry, rz);
                const bool flt = HALF ? h > thr : h != self;
                const bool in = (r2 < hi) & flt;
                tie |= in & !(r2 < lo);
                col[max(min(cnt, cap - 4), 0) * stride] = (unsigned short)h;
                cnt += in;
            }
        }
        // The walk kept every candidate below the upper edge of the FP32
        // rounding band of the list radius.  Where some kept candidate lies in
        // the band (rare), the list is compacted in place: the band's entries
        // stay only when the FP64 distance from the master positions is below
        // the list radius.  (A list that outgrew the stage is walked again
        // below, with the same decisions.)
        if (valid && tie && cnt <= cap - 4) {
            int kept = 0;
            for (int k = 0; k < cnt; ++k) {
                const int h = col[k * stride];
                bool keep = C::sep2(p, halo[h], ry, rz) < lo;
                if (!keep) {
                    int j = -1;
                    for (int r = 0; r < nrng; ++r) {
                        const int a = rng[half][r][0], e = rng[half][r][1];
                        if (h >= a && h < e) j = rng[half][r][2] + (h - a);
                    }
                    keep = j >= 0 && r2_fp64(X, b.S, i, j, R.L) < R.rl2;
                }
                if (keep) col[(kept++) * stride] = (unsigned short)h;
            }
            cnt = kept;
        }
        // a list longer than the stage allows (or a tile without a stage):
        // walk the candidates again in the same order; rows below cap go to
        // the stage, the rest to global memory
        if (valid && cnt > cap - 4) {
            int c2 = 0;
            auto put = [&](int h) {
                if (c2 < cap) lst[c2 * Pt + pp] = (unsigned short)h;
                else if (c2 < b.K) b.nbr[nbr_index(tl.s0, Pt, b.K, c2, pp)] = (unsigned short)h;
                ++c2;
            };
            for (int r = 0; r < nrng; ++r) {
                const int thr = HALF ? i - rng[half][r][2] + rng[half][r][0] : 0;
                for (int h = rng[half][r][0]; h < rng[half][r][1]; ++h) {
                    const float r2 = C::sep2(p, halo[h], ry, rz);
                    if ((r2 < lo) & (HALF ? h > thr : h != self)) put(h);
                }
            }
            if (tie)
                for (int r = 0; r < nrng; ++r) {
                    const int h0 = rng[half][r][0], h1 = rng[half][r][1], j0 = rng[half][r][2];
                    const int thr = HALF ? i - j0 + h0 : 0;
                    for (int h = h0; h < h1; ++h) {
                        const float r2 = C::sep2(p, halo[h], ry, rz);
                        if ((r2 < hi) & !(r2 < lo) & (HALF ? h > thr : h != self) &&
                            r2_fp64(X, b.S, i, j0 + (h - h0), R.L) < R.rl2)
                            put(h);
                    }
                }
            cnt = c2;   // the walk's count included band candidates that FP64 may reject
        }
        if (valid) {
            // pad with the particle's own index (r = 0 is never an interaction)
            const int kp = min(((cnt + kPad - 1) / kPad) * kPad, b.K);
            for (int k = cnt; k < kp; ++k) {
                if (k < cap) lst[k * Pt + pp] = (unsigned short)self;
                else b.nbr[nbr_index(tl.s0, Pt, b.K, k, pp)] = (unsigned short)self;
            }
            b.nn[i] = cnt;
            if (cnt > b.K) err |= kErrList;
            atomicMax(s_kmax, kp);
            mx = max(mx, cnt);
            sm += cnt;
        }
        __syncwarp();   // the range table is rewritten for the next group
    }
}

// The halo pieces (contiguous runs of 16-byte positions) by bulk (TMA)
// copies, issued by the 32 lanes of one warp in parallel (up to 18 pieces):
// lane 0 arms the staging barrier with the halo's byte count, then lane q
// issues piece q.
__device__ __forceinline__ void issue_halo_bulk_warp(const Piece *pc, int np, const uint4 *P, uint4 *halo,
                                                     unsigned long long *bar, int lane)
{
    if (lane == 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar, (unsigned)pc[np].hoff * 16u);
    }
    __syncwarp();
    fence_proxy_async_smem();
    if (lane < np && pc[lane].n > 0) bulk_g2s(&halo[pc[lane].hoff], &P[pc[lane].slot0], (unsigned)pc[lane].n * 16u, bar);
}

__global__ void __launch_bounds__(kBlock, 4) k_build_list(Bufs b)
{
    if (block_uniform(!b.ctl->rebuild || b.ctl->err)) return;
    extern __shared__ uint4 halo[];
    float4 *halof = reinterpret_cast<float4 *>(halo);                          // the same entries, converted
    unsigned short *lst = reinterpret_cast<unsigned short *>(halo + b.hcap);   // [k][Pt] stage, then 32 dummy slots
    // tile records and halo pieces, double-buffered: the next tile's are
    // copied in by one warp while this one is walked
    __shared__ Piece pcb[2][kMaxPieces + 1];
    __shared__ Tile tlb[2];
    __shared__ int s_npb[2];
    __shared__ int s_tile, s_kmax, s_next, s_issued;
    int buf = 0;
    bool have = false;
    __shared__ int s_rng[kBlock / 32][2][kMaxPieces][3];   // per warp: the ranges of both half-warp unions
    __shared__ __align__(8) unsigned long long s_mbar;     // completion of a tile's halo copies
    unsigned phase = 0;
    const int src = b.ctl->cur ^ 1;          // k_reorder wrote the sorted state here
    const uint4 *P = b.pos[src];
    const double *X = b.x[src];
    const int warp = threadIdx.x >> 5;
    int mx = 0;
    long long sm = 0;
    int err = 0;
    if (threadIdx.x == 0) {
        s_tile = (int)atomicAdd(&b.ctl->tile_next, 1u);
        s_issued = 0;
        mbar_init(&s_mbar, 1);
    }
    __syncthreads();
    for (;;) {
        const int t = s_tile;
        const bool issued = s_issued != 0;   // this tile's halo copies went out during the last one
        __syncthreads();
        if (t >= b.ctl->ntiles) break;
        // the next tile is claimed now and published at the end of this one
        int t_next = 0;
        if (threadIdx.x == 0) { t_next = (int)atomicAdd(&b.ctl->tile_next, 1u); s_kmax = 0; }
        if (!have) load_tile(b, t, tlb[buf], pcb[buf], s_npb[buf]);
        __syncthreads();
        const Piece *const pc = pcb[buf];
        const Tile &tl = tlb[buf];
        const int s_np = s_npb[buf];
        const Replica &R = b.rep[tl.rep];
        const int H = pc[s_np].hoff;
        const int Pt = tl.s1 - tl.s0;
        if (H > b.hcap) {
            err |= kErrList;                 // halo does not fit: the host grows hcap and rebuilds
            for (long long i = tl.s0 + threadIdx.x; i < tl.s1; i += blockDim.x) b.nn[i] = 0;
            if (threadIdx.x == 0) { s_tile = t_next; s_issued = 0; }
            __syncthreads();
            have = false;
            continue;
        }
        // the halo pieces (contiguous runs of 16-byte positions) by bulk (TMA)
        // copies issued by the first warp; every thread waits on the barrier
        if (threadIdx.x == 0) s_next = t_next;
        if (threadIdx.x < 32 && !issued) issue_halo_bulk_warp(pc, s_np, P, halo, &s_mbar, threadIdx.x);
        const bool late = !mbar_wait(&s_mbar, phase);
        phase ^= 1u;
        if (__syncthreads_or(late)) {   // a bulk copy never completed: stop, report
            err |= kErrTimeout;
            break;
        }
        // the last warp copies the next tile's record and pieces into the other
        // buffer while this one is walked
        const int tn = s_next;
        const bool pref = tn < b.ctl->ntiles;
        if (pref && threadIdx.x >= blockDim.x - 32)
            prefetch_tile_async(b, tn, tlb[buf ^ 1], pcb[buf ^ 1], s_npb[buf ^ 1], threadIdx.x & 31);
        const bool rel = R.ncell[1] >= 3 && R.ncell[2] >= 3 && tl.x1 - tl.x0 <= R.ncell[0] - 3;
        if (rel) {
            // FP32 coordinates relative to the tile centre (exact integer
            // minimum image, one rounding), y and z in x-axis units
            const unsigned cx = (unsigned)((((unsigned long long)(tl.x0 + tl.x1)) << 31) / (unsigned)R.ncell[0]);
            const unsigned cy = (unsigned)((((unsigned long long)(2 * tl.cy + 1)) << 31) / (unsigned)R.ncell[1]);
            const unsigned cz = (unsigned)((((unsigned long long)(2 * tl.cz + 1)) << 31) / (unsigned)R.ncell[2]);
#pragma unroll 4
            for (int h = threadIdx.x; h < H; h += blockDim.x) {
                const uint4 q = halo[h];
                halof[h] = make_float4((float)(int)(q.x - cx), (float)(int)(q.y - cy) * R.ry,
                                       (float)(int)(q.z - cz) * R.rz, __int_as_float(h));
            }
        }
        __syncthreads();
        const int hfirst = tile_self_offset(R, tl, pc, s_np);
        if (b.half_list) {
            if (rel) cells_of_tile<true, true>(b, R, tl, pc, s_np, halof, lst, X, hfirst, s_rng[warp], &s_kmax, mx, sm, err);
            else cells_of_tile<false, true>(b, R, tl, pc, s_np, halo, lst, X, hfirst, s_rng[warp], &s_kmax, mx, sm, err);
        } else {
            if (rel) cells_of_tile<true, false>(b, R, tl, pc, s_np, halof, lst, X, hfirst, s_rng[warp], &s_kmax, mx, sm, err);
            else cells_of_tile<false, false>(b, R, tl, pc, s_np, halo, lst, X, hfirst, s_rng[warp], &s_kmax, mx, sm, err);
        }
        cp_async_wait_all();   // the next tile's record (the copying warp)
        __syncthreads();
        // the halo is free: the next tile's halo copies go out now and arrive
        // while this tile's lists are copied out
        int issued_next = 0;   // the first warp (thread 0 publishes it)
        if (threadIdx.x == 0) b.tiles[t].kmax = s_kmax;
        if (threadIdx.x < 32 && pref) {
            const int npn = s_npb[buf ^ 1];
            if (pcb[buf ^ 1][npn].hoff <= b.hcap) {
                issue_halo_bulk_warp(pcb[buf ^ 1], npn, P, halo, &s_mbar, threadIdx.x);
                issued_next = 1;
            }
        }
        // the staged rows are the start of the tile's list block: one
        // contiguous copy (the block starts 64-byte aligned)
        const int cap = Pt <= kTileMax ? min((kListStage * kTileMax) / max(Pt, 1), b.K) : 0;
        const int total = min(s_kmax, cap) * Pt;
        unsigned short *dst = b.nbr + nbr_index(tl.s0, Pt, b.K, 0, 0);
        const uint4 *s4 = reinterpret_cast<const uint4 *>(lst);
        uint4 *d4 = reinterpret_cast<uint4 *>(dst);
        for (int m = threadIdx.x; m < (total >> 3); m += blockDim.x) d4[m] = s4[m];
        for (int m = ((total >> 3) << 3) + threadIdx.x; m < total; m += blockDim.x) dst[m] = lst[m];
        if (threadIdx.x == 0) {
            s_tile = t_next;
            s_issued = issued_next;
        }
        __syncthreads();
        buf ^= 1;
        have = pref;
    }
    if (err) atomicOr(&b.ctl->err, err);
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        sm += __shfl_xor_sync(0xffffffffu, sm, o);
    }
    if ((threadIdx.x & 31) == 0 && sm > 0) {
        atomicMax(&b.ctl->max_nn, mx);
        atomicAdd((unsigned long long *)&b.ctl->list_entries, (unsigned long long)sm);
    }
    // last block: publish the sorted buffers and clear the rebuild decision
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned prev = atomicAdd(&b.ctl->done_list, 1u);
        if (prev == gridDim.x - 1) {
            __threadfence();
            b.ctl->cur ^= 1;
            b.ctl->rebuild = 0;
            b.ctl->disp2_bits = 0u;
            b.ctl->rebuilds += 1;
            b.ctl->done_list = 0u;
            b.ctl->tile_next = 0u;
        }
    }
}

// ---------------------------------------------------------------- pair export
__global__ void k_export_pairs(Bufs b, int *pairs, long long cap, unsigned long long *count)
{
    __shared__ Piece pc[kMaxPieces + 1];
    __shared__ int s_np;
    const uint4 *P = b.pos[b.ctl->cur];
    for (int t = blockIdx.x; t < b.ctl->ntiles; t += gridDim.x) {
        __syncthreads();
        const Tile tl = b.tiles[t];
        const Replica &R = b.rep[tl.rep];
        (void)R;
        if (threadIdx.x == 0) s_np = b.tile_np[t];
        for (int m = threadIdx.x; m <= kMaxPieces; m += blockDim.x) pc[m] = b.pieces[(size_t)t * (kMaxPieces + 1) + m];
        __syncthreads();
        const int Pt = tl.s1 - tl.s0;
        for (long long i = tl.s0 + threadIdx.x; i < tl.s1; i += blockDim.x) {
            const int idi = (int)P[i].w;
            const int n = min(b.nn[i], b.K);
            for (int k = 0; k < n; ++k) {
                const int h = b.nbr[nbr_index(tl.s0, Pt, b.K, k, (int)(i - tl.s0))];
                int q = 0;
                while (q + 1 < s_np && h >= pc[q + 1].hoff) ++q;
                const int j = pc[q].slot0 + (h - pc[q].hoff);
                const int idj = (int)P[j].w;
                // a full list holds every pair twice (kept once, from its
                // lower id), a half list once (exported as (lower, higher))
                if (b.half_list || idi < idj) {
                    unsigned long long w = atomicAdd(count, 1ull);
                    if ((long long)w < cap) { pairs[2 * w] = min(idi, idj); pairs[2 * w + 1] = max(idi, idj); }
                }
            }
        }
    }
}

// ---------------------------------------------------------------- launchers
static inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

void launch_set_state(const Bufs &b, const double *x, const double *v, cudaStream_t st)
{
    k_reset_ctl<<<1, 1, 0, st>>>(b.ctl);
    k_set_state<<<b.nblk, kBlock, 0, st>>>(b, x, v);
}

void launch_get_state(const Bufs &b, double *x, double *v, cudaStream_t st)
{
    k_get_state<<<b.nblk, kBlock, 0, st>>>(b, x, v);
}

void launch_set_rebuild(const Bufs &b, cudaStream_t st) { k_set_rebuild<<<1, 1, 0, st>>>(b.ctl); }

void launch_reload(const Bufs &b, const double *x, cudaStream_t st)
{
    k_reload<<<b.nblk, kBlock, 0, st>>>(b, x);
    k_reload_decide<<<1, 1, 0, st>>>(b.ctl);
}

void launch_cond(const Bufs &b, unsigned long long handle, int what, cudaStream_t st)
{
    k_cond<<<1, 1, 0, st>>>(b.ctl, (cudaGraphConditionalHandle)handle, what);
}

void launch_force_by_id(const Bufs &b, double *buf, int dir, cudaStream_t st)
{
    k_force_by_id<<<(unsigned)((b.S + 255) / 256), 256, 0, st>>>(b, buf, dir);
}
void launch_set_steps(const Bufs &b, long long left, cudaStream_t st) { k_set_steps<<<1, 1, 0, st>>>(b.ctl, left); }

void launch_record_x(const Bufs &b, cudaStream_t st) { k_record_x<<<b.nblk, kBlock, 0, st>>>(b); }

static int list_grid(size_t smem)
{
    static int grid = 0;
    static size_t grid_smem = 0;
    if (grid == 0 || grid_smem != smem) {
        int dev = 0, nsm = 0, occ = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        // the default 48 KB limit covers static plus dynamic shared memory: always opt in
        cudaFuncSetAttribute((const void *)k_build_list, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void *)k_build_list, kBlock, smem);
        grid = (occ > 0 ? occ : 1) * (nsm > 0 ? nsm : 1);
        grid_smem = smem;
    }
    return grid;
}

// blocks of the bounded-grid chain kernels: 16 per SM, at most `need`
static unsigned chain_grid(long long need)
{
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm <= 0) nsm = 1;
    }
    const long long cap = 16LL * nsm;
    return (unsigned)(need < cap ? (need > 0 ? need : 1) : cap);
}

void launch_rebuild_chain(const Bufs &b, cudaStream_t st)
{
    k_bin<<<chain_grid(b.nblk), kBlock, 0, st>>>(b);
    const unsigned nsb = (unsigned)((b.C + kScanBlock - 1) / kScanBlock);
    k_scan_sum<<<nsb, kScanBlock, 0, st>>>(b);
    k_scan_top<<<1, kScanThreads, 0, st>>>(b);
    k_scan_write<<<nsb, kScanBlock, 0, st>>>(b);
    k_scatter<<<chain_grid(b.nblk), kBlock, 0, st>>>(b);
    k_reorder<<<chain_grid(blocks_for((long long)b.C * 8, 256)), 256, 0, st>>>(b);
    const long long nt = b.n_bond_ent > b.n_ang_ent ? b.n_bond_ent : b.n_ang_ent;
    if (nt > 0) k_topology_slots<<<blocks_for(nt, 256), 256, 0, st>>>(b);
    k_tile_count<<<blocks_for(b.nrows, kTileWarps), 32 * kTileWarps, 0, st>>>(b);
    k_tile_scan<<<1, kScanThreads, 0, st>>>(b);
    k_tile_write<<<blocks_for(b.nrows, kTileWarps), 32 * kTileWarps, 0, st>>>(b);
    k_tile_pieces<<<chain_grid(blocks_for(b.C, kTileWarps)), 32 * kTileWarps, 0, st>>>(b);
    const size_t smem = list_smem_bytes(b.hcap);
    k_build_list<<<list_grid(smem), kBlock, smem, st>>>(b);
}

void launch_export_pairs(const Bufs &b, int *pairs, long long cap, unsigned long long *count, cudaStream_t st)
{
    k_export_pairs<<<1024, kBlock, 0, st>>>(b, pairs, cap, count);
}

}  // namespace mdk
