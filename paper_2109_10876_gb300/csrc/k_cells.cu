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
    long long q = __double2ll_rn(y * scale);
    return (unsigned)(q & 0xffffffffLL);
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
__device__ __forceinline__ double r2_fp64(const double *x, long long S, long long i, long long j,
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
    ctl->max_occ = ctl->max_nn = 0;
    ctl->step = 0;
    ctl->rebuilds = 0;
    ctl->list_entries = 0;
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

// ---------------------------------------------------------------- counting sort
// a1: cell id of every particle and the cell histogram.
__global__ void k_bin(Bufs b)
{
    if (!b.ctl->rebuild || b.ctl->err) return;
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.S) return;
    uint4 p = b.pos[b.ctl->cur][s];
    if ((int)p.w < 0) return;
    const Replica &R = b.rep[b.blk_rep[blockIdx.x]];
    int cx, cy, cz;
    cell_coords(p, R, cx, cy, cz);
    int c = R.cell_off + (cz * R.ncell[1] + cy) * R.ncell[0] + cx;
    b.cellid[s] = c;
    atomicAdd(&b.cell_count[c], 1);
}

// Exclusive scan of the histogram, per replica, offset by the replica's first
// slot.  One block of 1024 threads; each thread scans a contiguous chunk.
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

__global__ void __launch_bounds__(kScanThreads) k_scan(Bufs b)
{
    if (!b.ctl->rebuild || b.ctl->err) return;
    __shared__ int warp_sums[33];
    if (threadIdx.x == 0) {
        b.ctl->max_nn = 0;
        b.ctl->list_entries = 0;
        b.ctl->max_occ = 0;
    }
    int local_max = 0;
    for (int r = 0; r < b.nrep; ++r) {
        const Replica &R = b.rep[r];
        int n = R.ncells;
        int chunk = (n + kScanThreads - 1) / kScanThreads;
        int lo = min(n, (int)threadIdx.x * chunk), hi = min(n, lo + chunk);
        int sum = 0;
        for (int c = lo; c < hi; ++c) {
            int k = b.cell_count[R.cell_off + c];
            sum += k;
            local_max = max(local_max, k);
        }
        int total;
        int base = block_excl_scan(sum, warp_sums, total) + (int)R.slot_begin;
        for (int c = lo; c < hi; ++c) {
            int k = b.cell_count[R.cell_off + c];
            b.cell_start[R.cell_off + c] = base;
            b.cell_end[R.cell_off + c] = base;   // cursor for the scatter
            base += k;
        }
    }
    for (int o = 16; o > 0; o >>= 1) local_max = max(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&b.ctl->max_occ, local_max);
}

// Scatter each particle's old slot into its cell's bucket (order within a
// cell is fixed afterwards by k_reorder).
__global__ void k_scatter(Bufs b)
{
    if (!b.ctl->rebuild || b.ctl->err) return;
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.S) return;
    if ((int)b.pos[b.ctl->cur][s].w < 0) return;
    int c = b.cellid[s];
    int k = atomicAdd(&b.cell_end[c], 1);
    b.bucket[k] = (int)s;
}

// One warp per cell: order the cell's members by particle id (so the slot
// order is a function of the positions alone), then gather x, v, pos from
// buffer cur into buffer cur ^ 1 at the new slots.
__global__ void k_reorder(Bufs b)
{
    if (!b.ctl->rebuild || b.ctl->err) return;
    long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (gw >= b.C) return;
    int c = (int)gw;
    int start = b.cell_start[c], end = b.cell_end[c];
    int n = end - start;
    if (lane == 0) b.cell_count[c] = 0;   // histogram is clean for the next build
    int cur = b.ctl->cur, nxt = cur ^ 1;
    const uint4 *pin = b.pos[cur];
    for (int m = lane; m < n; m += 32) {
        int s = b.bucket[start + m];
        uint4 p = pin[s];
        int id = (int)p.w;
        int rank = 0;
        for (int q = 0; q < n; ++q) {
            int o = (int)pin[b.bucket[start + q]].w;
            rank += (o < id);
        }
        int dst = start + rank;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            b.x[nxt][k * b.S + dst] = b.x[cur][k * b.S + s];
            b.v[nxt][k * b.S + dst] = b.v[cur][k * b.S + s];
        }
        b.pos[nxt][dst] = p;
        b.xref[dst] = p;
        b.slot_of_id[id] = dst;
        b.cellid[dst] = c;
    }
}

// a2: Verlet list of every pair within r_cut + r_skin, one thread per slot,
// scanning the own cell and its neighbours.  The FP32 distance decides all
// pairs except those within its rounding of the list radius, which are
// settled in FP64 from the master positions (same formula as the FP64
// reference), so the list is exactly the FP64 pair set.
__device__ __forceinline__ void stencil(int n, int &lo, int &cnt)
{
    // unique neighbour offsets along an axis with n cells
    if (n >= 3) { lo = -1; cnt = 3; }
    else if (n == 2) { lo = 0; cnt = 2; }
    else { lo = 0; cnt = 1; }
}

__global__ void __launch_bounds__(kBlock) k_build_list(Bufs b)
{
    if (!b.ctl->rebuild || b.ctl->err) return;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int src = b.ctl->cur ^ 1;            // k_reorder wrote the sorted state here
    const Replica &R = b.rep[b.blk_rep[blockIdx.x]];
    int cnt = 0;
    bool real = false;
    if (i < b.S) {
        uint4 p = b.pos[src][i];
        real = (int)p.w >= 0;
        if (real) {
            int c = b.cellid[i] - R.cell_off;
            int cx = c % R.ncell[0], cy = (c / R.ncell[0]) % R.ncell[1], cz = c / (R.ncell[0] * R.ncell[1]);
            int lx, nx, ly, ny, lz, nz;
            stencil(R.ncell[0], lx, nx);
            stencil(R.ncell[1], ly, ny);
            stencil(R.ncell[2], lz, nz);
            const uint4 *P = b.pos[src];
            const double *X = b.x[src];
            for (int oz = 0; oz < nz; ++oz) {
                int zz = cz + lz + oz;
                zz += (zz < 0) ? R.ncell[2] : 0;
                zz -= (zz >= R.ncell[2]) ? R.ncell[2] : 0;
                for (int oy = 0; oy < ny; ++oy) {
                    int yy = cy + ly + oy;
                    yy += (yy < 0) ? R.ncell[1] : 0;
                    yy -= (yy >= R.ncell[1]) ? R.ncell[1] : 0;
                    for (int ox = 0; ox < nx; ++ox) {
                        int xx = cx + lx + ox;
                        xx += (xx < 0) ? R.ncell[0] : 0;
                        xx -= (xx >= R.ncell[0]) ? R.ncell[0] : 0;
                        int cn = R.cell_off + (zz * R.ncell[1] + yy) * R.ncell[0] + xx;
                        int j0 = b.cell_start[cn], j1 = b.cell_end[cn];
                        for (int j = j0; j < j1; ++j) {
                            if (j == i) continue;
                            float r2 = r2_q(p, P[j], R.qs);
                            bool in = r2 < R.rl2_lo;
                            if (!in && r2 < R.rl2_hi) in = r2_fp64(X, b.S, i, j, R.L) < R.rl2;
                            if (in) {
                                if (cnt < b.K) b.nbr[nbr_index(i, cnt, b.K)] = j;
                                ++cnt;
                            }
                        }
                    }
                }
            }
        }
        b.nn[i] = cnt;
    }
    if (cnt > b.K) atomicOr(&b.ctl->err, kErrList);
    // block reduction of max and sum of list lengths
    int mx = cnt, sm = cnt;
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
        }
    }
}

// ---------------------------------------------------------------- pair export
__global__ void k_export_pairs(Bufs b, int *pairs, long long cap, unsigned long long *count)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.S) return;
    const uint4 *P = b.pos[b.ctl->cur];
    int idi = (int)P[i].w;
    if (idi < 0) return;
    int n = min(b.nn[i], b.K);
    for (int k = 0; k < n; ++k) {
        int j = b.nbr[nbr_index(i, k, b.K)];
        int idj = (int)P[j].w;
        if (idi < idj) {
            unsigned long long q = atomicAdd(count, 1ull);
            if ((long long)q < cap) { pairs[2 * q] = idi; pairs[2 * q + 1] = idj; }
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

void launch_rebuild_chain(const Bufs &b, cudaStream_t st)
{
    k_bin<<<b.nblk, kBlock, 0, st>>>(b);
    k_scan<<<1, kScanThreads, 0, st>>>(b);
    k_scatter<<<b.nblk, kBlock, 0, st>>>(b);
    k_reorder<<<blocks_for((long long)b.C * 32, 256), 256, 0, st>>>(b);
    k_build_list<<<b.nblk, kBlock, 0, st>>>(b);
}

void launch_export_pairs(const Bufs &b, int *pairs, long long cap, unsigned long long *count, cudaStream_t st)
{
    k_export_pairs<<<b.nblk, kBlock, 0, st>>>(b, pairs, cap, count);
}

}  // namespace mdk
