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
//   nbr, nn        Verlet list in warp slices: the lists of slots 32w .. 32w+31
//                  form one contiguous block of K rows of 32 entries, entry k of
//                  slot s at nbr[(s / 32) * 32 K + 32 k + s % 32]; nn[s] entries.
//                  A warp reads its 32 lists as one contiguous stream.
//   cells          count / start / end per cell of every replica grid.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mdk {

constexpr int kBlock = 128;          // threads per block of the per-slot kernels
constexpr int kMaxReplicas = 4096;

// error bits latched in Ctl::err
enum : int {
    kErrList = 1,
    kErrNonfinite = 2,
    kErrBond = 4,
    kErrFixed = 8,
    kErrTimeout = 16,
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
    long long slot_begin; // first slot
    long long n;          // real particles
    long long id_begin;   // first particle id (caller numbering)
    int blk_begin, blk_end;
    // pair potential (Eq. 2), FP64 and FP32 copies
    double eps, sigma, rc, rc2, vshift;   // vshift = V(rc) (0 shift for none)
    double rl2;                           // (r_cut + r_skin)^2
    float eps24_f, sig2_f, rc2_f, vshift_f, eps4_f;
    float rc2_lo, rc2_hi;                 // FP32 band around rc^2 resolved in FP64
    float rl2_lo, rl2_hi;                 // FP32 band around (r_cut + r_skin)^2
    float disp2_thr;                      // (r_skin / 2)^2, minus a margin
    float fmax2;                          // largest r^-2 (smallest r) the fixed-point range covers
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
    int pad0;
    long long step;          // index of the current positions x_step
    long long rebuilds;
    long long list_entries;
};

// index of entry k of slot s in the sliced list
__host__ __device__ __forceinline__ long long nbr_index(long long s, int k, int K)
{
    return (s >> 5) * (32LL * K) + 32LL * k + (s & 31);
}

// Everything the kernels touch.  Plain pointers; sizes in slots S, cells C,
// list capacity K per slot, particles N.
struct Bufs {
    double *x[2];
    double *v[2];
    uint4 *pos[2];
    double *F;               // stored total force of the current state, 3 * S, slot order
    uint4 *xref;
    int *slot_of_id;         // N
    int *cellid;             // S
    int *cell_count;         // C
    int *cell_start;         // C
    int *cell_end;           // C (cursor during the scatter, then one past the last slot)
    int *bucket;             // S
    int *nbr;                // K * S
    int *nn;                 // S
    const Replica *rep;      // n_rep
    const int *blk_rep;      // replica of every block of kBlock slots
    const int *bond_off;     // N + 1, bonds of particle id (both directions)
    const int *bond_partner; // 2 * n_bonds particle ids
    double *partial;         // 4 per block: U, K, W partial sums
    double *thermo;          // where the last block writes (U, K, W) per replica, or null
    double *fout;            // force output in caller order (3 * N) or null
    Ctl *ctl;
    long long S, N;
    int C, K, nrep, nblk;
    int has_bonds;
    int langevin;
    double dt, mass, half_dt_over_m;
    double gamma, kT, noise_amp;  // noise_amp = sqrt(24 gamma kT m / dt)
    double fene_K, fene_R02;
    float fene_K_f, fene_R02_f;
    unsigned long long seed;
};

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
void launch_export_pairs(const Bufs &b, int *pairs, long long cap, unsigned long long *count, cudaStream_t st);
void launch_set_rebuild(const Bufs &b, cudaStream_t st);

}  // namespace mdk
