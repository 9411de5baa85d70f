// Internal declarations shared by the CUDA translation units of the library.
//
// State layout in HBM (slot order = particles sorted by (replica, cell, id);
// S = total slots, each replica's slot range padded to a multiple of kBlock
// so that no thread block straddles two replicas):
//   x[2], v[2]     FP64, 3 * S, component-major (x[k * S + s]); double-buffered:
//                  a drift or a re-sort reads buffer `cur` and writes `cur ^ 1`.
//   pos[2]         uint4 per slot: 32-bit fixed-point coordinates
//                  q_k = round(x_k * 2^32 / L_k) mod 2^32 and, in .w, the
//                  particle id (-1 for padding).  The difference of two q's as
//                  int32 is the minimum-image separation in units of L_k / 2^32,
//                  exact, with the periodic wrap done by integer overflow.
//   xref           uint4 per slot: pos at the last list build (displacement check).
//   tiles          runs of consecutive cells along an x-row of a replica grid,
//                  cut at every rebuild so that a tile holds at most kTileMax
//                  particles and its halo (the tile's cells widened by one cell
//                  in x, on the 3 x 3 neighbouring rows) at most Hcap particles.
//                  A tile's particles are one contiguous slot range; its halo
//                  is a fixed sequence of contiguous slot ranges ("pieces").
//   nbr, nn        Verlet list of 16-bit halo indices, by tile: the lists of a
//                  tile's P = s1 - s0 particles occupy nbr[s0 K, s1 K) as K rows
//                  of P entries, entry k of particle p = s - s0 at
//                  nbr[s0 K + k P + p]; the threads of a tile read a row as one
//                  contiguous run.  nn[s] entries, padded with the particle's
//                  own halo index up to a multiple of kPad.
//   cells          count / start / end per cell of every replica grid.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mdk {

constexpr int kBlock = 128;          // threads per block of the per-slot kernels
constexpr int kMaxReplicas = 4096;
constexpr int kTileMax = 128;        // particles per tile (one per thread)
constexpr int kScanBlock = 1024;     // cells per block of the cell scan
constexpr int kMaxPieces = 18;       // 3 x 3 rows, at most 2 x-pieces each

// error bits latched in Ctl::err
enum : int {
    kErrList = 1,
    kErrNonfinite = 2,
    kErrBond = 4,
    kErrFixed = 8,
    kErrTimeout = 16,
    kErrBounds = 32,     // a device-side bounds check failed (checked build only)
};

// Sites of the device-side bounds checks of the checked build: each names an
// index that the data layout keeps in range by construction.
enum CheckSite : int {
    kSiteNone = 0,
    kSiteBinCell = 1,      // k_bin: a particle's cell within its replica's cells
    kSiteScatter = 2,      // k_scatter: a bucket slot within its cell's slots
    kSiteReorder = 3,      // k_reorder: the particle id and the destination slot
    kSiteTopology = 4,     // k_topology_slots: bond and angle partner ids
    kSiteTileWrite = 5,    // tiling: a tile's index within the tile table
    kSitePieces = 6,       // k_tile_pieces: a tile's piece count within kMaxPieces
    kSiteListRange = 7,    // list build: a candidate range within the staged halo
    kSiteListSelf = 8,     // list build: a particle's own halo entry within the halo
    kSiteForceHalo = 9,    // force kernels: a list entry within the staged halo
    kSiteForceOwn = 10,    // force kernels: a particle's own halo entry within the halo
    kSiteForceSlot = 11,   // force kernels: the slot behind a halo entry within the slots
    kSiteBondSlot = 12,    // force kernel: a bond or angle partner's slot within the slots
    kSiteAdjHalo = 13,     // reverse pass: a list entry within the staged halo, an id or slot in range
    kSiteCount = 14,
};

// Per-replica constants (device copy written once at create time).
struct Replica {
    double L[3];          // box edges
    double to_q[3];       // 2^32 / L  (length -> fixed-point units)
    double from_q[3];     // L / 2^32
    float qs[3];          // L / 2^32 as float
    int ncell[3];         // cell grid, edge L / ncell >= r_cut + r_skin
    int cell_off;         // first global cell index of this replica
    int ncells;
    int row_off;          // first global row (rows = (cy, cz) pairs, cz-major)
    long long slot_begin; // first slot
    long long n;          // real particles
    long long id_begin;   // first particle id (caller numbering)
    int blk_begin, blk_end;
    // pair potential (Eq. 2), FP64 and FP32 copies
    double eps, sigma, rc, rc2, vshift;   // vshift = V(rc) (0 shift for none)
    double rl2;                           // (r_cut + r_skin)^2
    int soft;                             // cosine push-off instead of Eq. 2 (FP64 path only)
    float eps24_f, sig2_f, rc2_f, vshift_f, eps4_f;
    float rc2_lo, rc2_hi;                 // FP32 band around rc^2 resolved in FP64
    float rl2_lo, rl2_hi;                 // FP32 band around (r_cut + r_skin)^2
    float disp2_thr;                      // (r_skin / 2)^2, minus a margin
    float fmax2;                          // smallest r^2 the fixed-point range covers
    // the same constants with lengths in fixed-point units of the x axis
    // (u = L_x / 2^32), used by the FP32 pair loop: r2 and d stay in u
    int cubic;                            // all box edges equal: no per-axis scaling
    float ry, rz;                         // L_y / L_x, L_z / L_x
    float rc2_lo_u, rc2_hi_u, fmax2_u, sig2_u, eps24_u, rl2_lo_u, rl2_hi_u;
    float rl_win_u;                       // x-window half-width of the list walk (> r_list, in u)
};

// Device control block: every per-step decision lives here, so a step needs
// no host round trip and can be captured in a CUDA graph.
struct Ctl {
    int cur;                 // current buffer of x, v, pos
    int rebuild;             // 1: the next re-sort + list build must run
    unsigned disp2_bits;     // max squared displacement since the build (float bits)
    int err;                 // latched kErr* bits
    unsigned done_force;     // block-completion counters (last-block pattern)
    unsigned done_list;
    unsigned done_kick;
    int max_occ;             // largest cell occupancy at the last build
    int max_nn;              // longest list at the last build
    int ntiles;              // tiles of the current build
    unsigned tile_next;      // work counter of the persistent tile kernels
    int max_halo;            // largest halo of the current build
    long long step;          // index of the current positions x_step
    long long steps_left;    // fused steps still to run in a graph-launched md_step
    long long rec;           // energy records written by this graph-launched md_step
    long long rebuilds;
    long long list_entries;
    int bad_site;            // checked build: the first failing bounds check (CheckSite), else 0
    int plant;               // checked build: a site whose next checks are made to fail (self-test), else 0
    long long bad_index;     // checked build: the index that failed at bad_site
    long long step0;         // Ctl::step at the start of a graph-launched md_step (set by k_set_steps)
};

#ifdef MD_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

// A device-side bounds check.  In the default build it is `true` and
// compiles away.  Built with -DMD_CHECKED it returns `ok`; on a failure it
// latches kErrBounds, with the first failing site and index in the control
// block, and the caller replaces the access by a harmless one: nothing traps,
// so the context stays usable and the host reports MD_ERR_BOUNDS.  A site
// named by Ctl::plant fails on purpose (with an index in range), so that a
// test can exercise every site's failure path without a bad access.
__device__ __forceinline__ bool md_ok(Ctl *ctl, bool ok, int site, long long idx)
{
    if constexpr (!kChecked) {
        return true;
    } else {
        ok = ok && ctl->plant != site;
        if (!ok) {
            if (atomicCAS(&ctl->bad_site, 0, site) == 0) ctl->bad_index = idx;
            atomicOr(&ctl->err, kErrBounds);
        }
        return ok;
    }
}

// A tile: row (cy, cz) of replica rep, cells [x0, x1) along x, particles in
// slots [s0, s1), halo of hsize particles.
struct Tile {
    int rep, cy, cz, x0, x1, s0, s1, hsize;
    int kmax;   // longest padded list of the tile (written by the list build)
};

constexpr int kListStage = 96;       // list rows of a full tile staged in shared memory (x kTileMax entries)

// One contiguous slot range of a halo: cells [xa, xb) of halo row `row`,
// placed at halo offset hoff.
struct Piece {
    int row, xa, xb, slot0, hoff, n;
};

// Unique neighbour offsets along an axis with n cells: {-1, 0, 1}, {0, 1} or {0}.
__host__ __device__ __forceinline__ void axis_offsets(int n, int &lo, int &cnt)
{
    if (n >= 3) { lo = -1; cnt = 3; }
    else if (n == 2) { lo = 0; cnt = 2; }
    else { lo = 0; cnt = 1; }
}

__host__ __device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// Pieces of the halo of cells [x0, x1) on row (cy, cz): for each of the (up
// to) 3 x 3 rows in (dz, dy) order, the cells [x0 - 1, x1] along x (the whole
// row when that covers it), split at the periodic boundary.  Returns the
// number of pieces; fills p[] with their slot ranges and halo offsets.
__device__ __forceinline__ int halo_pieces(const int *cell_start, const int *cell_end, int cell_off,
                                           const int ncell[3], int cy, int cz, int x0, int x1, Piece *p,
                                           int *hsize = nullptr)
{
    const int nx = ncell[0], ny = ncell[1], nz = ncell[2];
    int ly, cntY, lz, cntZ;
    axis_offsets(ny, ly, cntY);
    axis_offsets(nz, lz, cntZ);
    int np = 0, h = 0, row = 0;
    for (int oz = 0; oz < cntZ; ++oz) {
        const int zz = wrapi(cz + lz + oz, nz);
        for (int oy = 0; oy < cntY; ++oy, ++row) {
            const int yy = wrapi(cy + ly + oy, ny);
            const int base = cell_off + (zz * ny + yy) * nx;
            int ra[2], rb[2], nr = 0;
            if (x1 - x0 + 2 >= nx) { ra[0] = 0; rb[0] = nx; nr = 1; }
            else if (x0 == 0) { ra[0] = nx - 1; rb[0] = nx; ra[1] = 0; rb[1] = x1 + 1; nr = 2; }
            else if (x1 == nx) { ra[0] = x0 - 1; rb[0] = nx; ra[1] = 0; rb[1] = 1; nr = 2; }
            else { ra[0] = x0 - 1; rb[0] = x1 + 1; nr = 1; }
            for (int q = 0; q < nr; ++q) {
                const int s0 = cell_start[base + ra[q]];
                const int n = cell_end[base + rb[q] - 1] - s0;
                if (p) { p[np].row = row; p[np].xa = ra[q]; p[np].xb = rb[q]; p[np].slot0 = s0; p[np].hoff = h; p[np].n = n; }
                ++np;
                h += n;
            }
        }
    }
    if (p) p[np].hoff = h;   // total halo size after the last piece
    if (hsize) *hsize = h;
    return np;
}

constexpr int kPad = 4;              // lists are padded to a multiple of this

// index of entry k of the particle p of a tile starting at slot s0 with P particles
__host__ __device__ __forceinline__ long long nbr_index(long long s0, int P, int K, int k, int p)
{
    return s0 * K + (long long)k * P + p;
}

// Everything the kernels touch.  Plain pointers; sizes in slots S, cells C,
// list capacity K per slot, particles N.
struct Bufs {
    double *x[2];
    double *v[2];
    uint4 *pos[2];
    double *F;               // stored total force of the current state, 3 * S, slot order
    long long *Fq;           // half list: 64-bit fixed-point force sums (3 * S, slot order), zero between steps
    long long *eacc;         // FP32 path: per-replica energy sums (4 * nrep: U, K, W, unused; twice the
                             // energies in units of 2^-22), zero between launches
    int half_list;           // 1: each pair once (Newton's third law), reactions by 64-bit atomics
    uint4 *xref;
    int *slot_of_id;         // N
    int *cellid;             // S
    int *cell_count;         // C
    int *cell_start;         // C
    int *cell_end;           // C (cursor during the scatter, then one past the last slot)
    const int *cell_pad;     // C: padding slots after a cell (the last cell of each replica)
    int *scan_part;          // blocks of the cell scan: their sums, then exclusive offsets
    int *row_rep;            // nrows: replica of every row (rows ordered by replica)
    int *bucket;             // S
    unsigned short *nbr;     // K * S halo indices
    int *nn;                 // S
    Tile *tiles;             // C (a tile has at least one cell)
    Piece *pieces;           // kMaxPieces + 1 per tile: the halo pieces, then the total in [np].hoff
    int *tile_np;            // pieces per tile
    int *row_tiles;          // rows: tiles per row, then their exclusive scan
    int *rep_tile;           // nrep + 1: first tile of every replica
    int nrows;               // rows over all replicas
    int hcap;                // halo capacity (particles) of the tile kernels
    int tile_max;            // particles per tile the tiler aims at (<= kTileMax; autotuned)
    const Replica *rep;      // n_rep
    const int *blk_rep;      // replica of every block of kBlock slots
    const int *bond_off;     // N + 1, bonds of particle id (both directions)
    const int *bond_partner; // 2 * n_bonds particle ids
    const int *ang_off;      // N + 1: angle entries of particle id
    const int4 *ang_ent;     // 3 * n_angles: (a, b, c, role of the particle: 0, 1, 2)
    float4 *adj_wa;          // reverse pass: w by slot as FP32 pieces (hi x, hi y, hi z, lo x), S entries
    float2 *adj_wb;          // (lo y, lo z), S entries
    int *bond_pslot;         // 2 * n_bonds: current slot of each bond_partner entry (refreshed per re-sort)
    int4 *ang_slot;          // 3 * n_angles: current slots of (a, b, c) and the role, per ang_ent entry
    long long n_bond_ent, n_ang_ent;
    int has_angles;
    double angle_K;
    float angle_K_f;
    double *partial;         // 4 per tile: U, K, W partial sums
    double *thermo;          // where the last block writes (U, K, W) per replica, or null
    double *thermo_ring;     // graph-launched md_step: record Ctl::rec goes to thermo_ring + 3 nrep rec
    double *fout;            // force output in caller order (3 * N) or null
    double *xring;           // positions recorded after every step of a graph-launched call: slot
                             // step - step0 at xring + 3 N (step - step0), caller order (or null)
    Ctl *ctl;
    long long S, N;
    int C, K, nrep, nblk;
    int has_bonds;
    int langevin;
    double dt, mass, half_dt_over_m;
    double half_dt_over_m_fix;   // half_dt_over_m * 2^-22 (exact): the kick factor of fixed-point forces
    double gamma, kT, noise_amp;  // noise_amp = sqrt(24 gamma kT m / dt)
    double fene_K, fene_R02;
    float fene_K_f, fene_R02_f;
    unsigned long long seed;
    unsigned long long g_while;  // graph conditional handle of the step loop (0 outside a graph)
};

// Asynchronous global -> shared copies (no register staging): every copy a
// block issues is in flight at once; cp_async_wait_all waits for this
// thread's copies (a hardware wait), to be followed by __syncthreads().
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}

// Bulk (TMA) copies global -> shared completing on an mbarrier (sm_90 and
// later): one thread arms the barrier with the byte count and issues the
// copies; every thread waits on the barrier's phase.  Addresses 16-byte
// aligned, sizes multiples of 16.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// a plain arrival (count 1, no bytes), release semantics at CTA scope
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// orders this thread's earlier generic-proxy accesses to shared memory before
// its later bulk copies into it
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Wait for the completion of the barrier phase with the given parity, giving
// up after `polls` polls (each may suspend the thread briefly; the default of
// 2^20 polls is about a second in all).  Returns false on giving up.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, int polls = (1 << 20))
{
    for (int it = 0; it < polls; ++it) {
        unsigned done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(smem_u32(bar)), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void prefetch_l1(const void *gmem)
{
    asm volatile("prefetch.global.L1 [%0];" ::"l"(gmem));
}

__device__ __forceinline__ void prefetch_l2(const void *gmem)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(gmem));
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Cooperative load of a tile record and its halo pieces into shared memory.
__device__ __forceinline__ void load_tile(const Bufs &b, int t, Tile &tl, Piece *pc, int &np)
{
    if (threadIdx.x == 0) { tl = b.tiles[t]; np = b.tile_np[t]; }
    const int *src = reinterpret_cast<const int *>(b.pieces + (size_t)t * (kMaxPieces + 1));
    int *dst = reinterpret_cast<int *>(pc);
    constexpr int words = (kMaxPieces + 1) * sizeof(Piece) / sizeof(int);
    for (int m = threadIdx.x; m < words; m += blockDim.x) dst[m] = src[m];
}

// The same record and pieces, copied asynchronously by the 32 lanes of one
// warp (completion: cp_async_wait_all by those lanes, then a block barrier).
__device__ __forceinline__ void prefetch_tile_async(const Bufs &b, int t, Tile &tl, Piece *pc, int &np, int lane)
{
    const int *src = reinterpret_cast<const int *>(b.pieces + (size_t)t * (kMaxPieces + 1));
    int *dst = reinterpret_cast<int *>(pc);
    constexpr int words = (kMaxPieces + 1) * sizeof(Piece) / sizeof(int);
    for (int m = lane; m < words; m += 32) cp_async4(dst + m, src + m);
    const int *ts = reinterpret_cast<const int *>(b.tiles + t);
    int *td = reinterpret_cast<int *>(&tl);
    constexpr int tw = sizeof(Tile) / sizeof(int);
    for (int m = lane; m < tw; m += 32) cp_async4(td + m, ts + m);
    if (lane == 0) cp_async4(&np, b.tile_np + t);
}

// A decision taken by thread 0 and shared with the whole block, so that every
// thread of a block takes the same early return: an error latched by another
// block while this one starts cannot split it across its barriers.
__device__ __forceinline__ bool block_uniform(bool v)
{
    __shared__ int s_flag;
    if (threadIdx.x == 0) s_flag = v ? 1 : 0;
    __syncthreads();
    const bool r = s_flag != 0;
    __syncthreads();                    // before any later use of s_flag
    return r;
}

// Halo index of the tile's first particle.  The tile's own cells lie,
// contiguous, inside one piece of its own row (pieces split only at the
// periodic boundary, which a tile does not straddle).
__device__ __forceinline__ int tile_self_offset(const Replica &R, const Tile &tl, const Piece *pc, int np)
{
    int ly, cntY, lz, cntZ;
    axis_offsets(R.ncell[1], ly, cntY);
    axis_offsets(R.ncell[2], lz, cntZ);
    const int crow = (-lz) * cntY + (-ly);
    int q = 0;
    while (q + 1 < np && !(pc[q].row == crow && pc[q].slot0 <= tl.s0 &&
                           tl.s0 < pc[q].slot0 + pc[q].n + (pc[q].n == 0)))
        ++q;
    return pc[q].hoff + (tl.s0 - pc[q].slot0);
}

// 1/a for a normal, positive a: the hardware reciprocal approximation refined
// by two Newton-Raphson steps y <- y + y (1 - a y), each of which squares the
// relative error, so the result is within about an ulp of 1/a.
__device__ __forceinline__ double rcp_newton(double a)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(a));
    double e = __fma_rn(-a, y, 1.0);
    y = __fma_rn(y, e, y);
    e = __fma_rn(-a, y, 1.0);
    return __fma_rn(y, e, y);
}

// One 16-byte shared-memory load of a staged halo position (the compiler
// would otherwise split it when the fourth word is not used).
__device__ __forceinline__ uint4 lds128(const uint4 *p)
{
    uint4 q;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(q.x), "=r"(q.y), "=r"(q.z), "=r"(q.w) : "r"(a));
    return q;
}

// A tile's halo and list block by bulk (TMA) copies, issued by the 32 lanes of
// the first warp (the force kernel and the reverse pass): lane 0 arms the staging
// barrier with the tile's byte count, then lane q < np copies halo piece q (a
// contiguous run of 16-byte positions) and lane np the list block, if it fits
// the stage (64-byte aligned, read rounded up to 16 bytes; the list and the
// stage carry that slack).  The copies go out in parallel.
__device__ __forceinline__ void issue_tile_bulk(const Bufs &b, const Tile &tl, const Piece *pc, int np, const uint4 *P,
                                                uint4 *hpos, unsigned short *lst, unsigned long long *bar, int lane)
{
    const int Pt = tl.s1 - tl.s0;
    const unsigned lbytes = tl.kmax * Pt <= kListStage * kTileMax ? ((unsigned)(tl.kmax * Pt) * 2u + 15u) & ~15u : 0u;
    if (lane == 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar, (unsigned)pc[np].hoff * 16u + lbytes);
    }
    __syncwarp();
    fence_proxy_async_smem();
    if (lane < np) {
        if (pc[lane].n > 0) bulk_g2s(&hpos[pc[lane].hoff], &P[pc[lane].slot0], (unsigned)pc[lane].n * 16u, bar);
    } else if (lane == np && lbytes) {
        bulk_g2s(lst, b.nbr + nbr_index(tl.s0, Pt, b.K, 0, 0), lbytes, bar);
    }
}

// Exact conversions between FP64 and 64-bit integers by adding and removing
// 1.5 * 2^52, whose unit in the last place is 1 (valid for |value| < 2^51).
// They replace the integer <-> FP64 conversion instructions, which are slow
// on this part's narrow FP64 pipe.
constexpr double kRound52 = 6755399441055744.0;          // 1.5 * 2^52
constexpr long long kRound52Bits = 0x4338000000000000LL;

// round(y * scale) to nearest (ties to even), one rounding of the exact product
__device__ __forceinline__ long long fix_round(double y, double scale)
{
    return __double_as_longlong(__fma_rn(y, scale, kRound52)) - kRound52Bits;
}

// the double equal to v (exact)
__device__ __forceinline__ double ll_to_double(long long v)
{
    return __dsub_rn(__longlong_as_double(v + kRound52Bits), kRound52);
}

// Flat copy of a tile's halo (all loads independent): element h of piece q.
template <class T, class F>
__device__ __forceinline__ void stage_halo(const Piece *pc, int np, F load)
{
    const int H = pc[np].hoff;
    int q = 0;
    for (int h = threadIdx.x; h < H; h += blockDim.x) {
        while (h >= pc[q + 1].hoff) ++q;   // pieces in ascending halo order
        load(h, pc[q].slot0 + (h - pc[q].hoff));
    }
}

// kernel modes of the force kernel
enum Mode : int {
    kModeOut = 0,     // forces (conservative) to fout / F, energies on request; no integration
    kModeStore = 1,   // total force (with Langevin) into F, no integration
    kModeFused = 2,   // F(x_n); v += dt/2 m F (end of step n); v += dt/2m F; x += dt v (step n+1)
    kModeFinal = 3,   // F(x_n); v += dt/2m F; store F
};

// launchers (defined in the .cu files)
void launch_set_state(const Bufs &b, const double *x, const double *v, cudaStream_t st);
void launch_rebuild_chain(const Bufs &b, cudaStream_t st);
void launch_force(const Bufs &b, int precision, int mode, bool energy, cudaStream_t st);
void launch_kick_drift(const Bufs &b, cudaStream_t st);
void launch_get_state(const Bufs &b, double *x, double *v, cudaStream_t st);
void launch_force_by_id(const Bufs &b, double *buf, int dir, cudaStream_t st);
void launch_reload(const Bufs &b, const double *x, cudaStream_t st);
void launch_export_pairs(const Bufs &b, int *pairs, long long cap, unsigned long long *count, cudaStream_t st);
void launch_set_rebuild(const Bufs &b, cudaStream_t st);
// graph conditionals: set `handle` to (ctl->rebuild != 0) (what = 0) or (ctl->steps_left > 0) (what = 1)
void launch_cond(const Bufs &b, unsigned long long handle, int what, cudaStream_t st);
void launch_set_steps(const Bufs &b, long long left, cudaStream_t st);
// the current positions, in caller order, into slot Ctl::step - Ctl::step0 of b.xring
void launch_record_x(const Bufs &b, cudaStream_t st);
// one block waiting on a barrier that nothing completes, `polls` polls at most
void launch_wait_selftest(const Bufs &b, int polls, cudaStream_t st);
void launch_adj_hvp(const Bufs &b, int precision, const double *w, double *hv, double scale, double *g,
                    cudaStream_t st);
void launch_adj_loss(const Bufs &b, const double *coef, double *lx, double *lv, double *sums, cudaStream_t st);
void launch_adj_finish_loss(const Bufs &b, const double *sums, const double *coef, double *g, cudaStream_t st);
void launch_adj_update(long long n3, double *lx, double *lv, const double *hv, double c, double dt, cudaStream_t st);
// lx += gx, lv += gv (either may be null)
void launch_adj_add(long long n3, double *lx, double *lv, const double *gx, const double *gv, cudaStream_t st);

}  // namespace mdk
