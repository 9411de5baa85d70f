// Pair forces over the Verlet list (Eq. 2 under r < r_cut, Sec. 2.1.1 of
// arXiv:2109.10876), FENE bonds and the Langevin force (Sec. 4), fused with
// the velocity-Verlet update (Fig. 1) and the energy / virial reductions.
//
// Two precisions:
//   FP32 + fixed point: separations come from the 32-bit fixed-point copies
//     of the positions (exact integer minimum image, one rounding to float);
//     the pair force is evaluated in FP32 and each component is split into two
//     exactly rounded integers, round(f) and round((f - round(f)) * 2^22), which
//     are summed in 32-bit integers.  The sum is the 64-bit fixed-point force
//     at resolution 2^-22, independent of summation order, and f_ij = -f_ji
//     holds bit for bit, so the forces of a closed system sum to exactly 0.
//     Pairs whose FP32 r^2 lies within rounding of r_cut^2 are decided in FP64
//     from the master positions, so the interacting set is the FP64 set.
//   FP64: the same sums in double precision from the master positions.
// Positions and velocities are integrated in FP64 in both precisions.
#include <math_constants.h>

#include "md_internal.cuh"

namespace mdk {

constexpr float kMagic = 12582912.0f;       // 1.5 * 2^23: x + kMagic rounds x to an integer
constexpr unsigned kMagicBits = 0x4B400000u;
constexpr float kFixScale = 4194304.0f;     // 2^22
constexpr double kFixInv = 1.0 / 4194304.0;
#ifndef MDK_FORCE_MIN_BLOCKS
#define MDK_FORCE_MIN_BLOCKS 4
#endif
constexpr int kU = kPad;                     // neighbours per batch: lists are padded to it

// Add round(a * c * 2^22) to the two-piece accumulator without rounding the
// product first: round(a c) from one FMA against kMagic, the remainder
// a c - round(a c) from a second FMA (|remainder| <= 1/2), then its 2^-22
// multiple.  A deterministic, odd function of (a, c): f_ij = -f_ji exactly.
// Valid for |a c| < 2^21.
__device__ __forceinline__ void fx_acc2(float a, float c, unsigned &hi, unsigned &lo)
{
    float t1 = __fmaf_rn(a, c, kMagic);           // kMagic + round(a c)
    float h = __fsub_rn(t1, kMagic);              // round(a c), exact
    float r = __fmaf_rn(a, c, -h);                // a c - round(a c)
    float t2 = __fmaf_rn(r, kFixScale, kMagic);   // kMagic + round(r 2^22)
    hi += __float_as_uint(t1) - kMagicBits;
    lo += __float_as_uint(t2) - kMagicBits;
}

// Two neighbours at once with the packed FP32 instructions of this part
// (each lane of a float2 rounds exactly as the scalar instruction does).  The
// integer pieces are added without their bias kMagicBits; the caller removes
// it once per term at the end (all sums are modulo 2^32, so this is exact).
__device__ __forceinline__ void fx_acc2x2(float2 a, float2 c, unsigned &hi, unsigned &lo)
{
    const float2 M = make_float2(kMagic, kMagic);
    const float2 t1 = __ffma2_rn(a, c, M);                                   // kMagic + round(a c)
    const float2 nh = __ffma2_rn(t1, make_float2(-1.0f, -1.0f), M);          // -round(a c), exact
    const float2 r = __ffma2_rn(a, c, nh);                                   // a c - round(a c)
    const float2 t2 = __ffma2_rn(r, make_float2(kFixScale, kFixScale), M);   // kMagic + round(r 2^22)
    hi += __float_as_uint(t1.x) + __float_as_uint(t1.y);
    lo += __float_as_uint(t2.x) + __float_as_uint(t2.y);
}

// Reciprocal by the hardware approximation (a pure function of its input).
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Add round(f * 2^22) to the two-piece accumulator (valid for |f| < 2^21).
__device__ __forceinline__ void fx_acc(float f, unsigned &hi, unsigned &lo)
{
    float t1 = __fadd_rn(f, kMagic);              // kMagic + round(f)
    float h = __fsub_rn(t1, kMagic);              // round(f), exact
    float r = __fsub_rn(f, h);                    // f - round(f), exact, |r| <= 1/2
    float t2 = __fmaf_rn(r, kFixScale, kMagic);   // kMagic + round(r * 2^22)
    hi += __float_as_uint(t1) - kMagicBits;
    lo += __float_as_uint(t2) - kMagicBits;
}

// round(f 2^22) by the exact two-integer split
__device__ __forceinline__ long long fx_round(float f)
{
    unsigned h = 0, l = 0;
    fx_acc(f, h, l);
    return (long long)(int)h * 4194304LL + (long long)(int)l;
}

__device__ __forceinline__ double wrap1(double y, double L)
{
    if (y >= L) y = y - L;
    if (y < 0.0) {
        y = y + L;
        if (y >= L) y = 0.0;
    }
    return y;
}

// FP64 minimum-image r^2 with the fixed rounding sequence of the reference
// (t = xi - xj; t -= L * rint(t / L); r2 = (dx^2 + dy^2) + dz^2).
__device__ __noinline__ double r2_exact(const double *x, long long S, long long i, long long j,
                                           const double *L)
{
    double d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double t = __dsub_rn(x[k * S + i], x[k * S + j]);
        double q = rint(__ddiv_rn(t, L[k]));
        d[k] = __dsub_rn(t, __dmul_rn(L[k], q));
    }
    return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32 x 32 -> 64-bit
// products, key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// Langevin force -gamma m v + sqrt(24 gamma kT m / dt) u, u uniform in
// (-1/2, 1/2) from Philox keyed by the seed and counted by (id, step).
__device__ __forceinline__ void langevin(const Bufs &b, int id, long long step, const double v[3], double f[3])
{
    uint4 c = make_uint4((unsigned)id, (unsigned)(unsigned long long)step,
                         (unsigned)((unsigned long long)step >> 32), 0x4C414E47u);
    uint2 k = make_uint2((unsigned)b.seed, (unsigned)(b.seed >> 32));
    uint4 r = philox10(c, k);
    unsigned w[3] = {r.x, r.y, r.z};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        double u = ((double)w[q] + 0.5) * (1.0 / 4294967296.0) - 0.5;
        f[q] += -b.gamma * b.mass * v[q] + b.noise_amp * u;
    }
}

// Block-wide sum of three doubles in a fixed order; result valid in thread 0.
__device__ __forceinline__ void block_sum3(double &a, double &c, double &d, double (*sm)[3])
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
        d += __shfl_down_sync(0xffffffffu, d, o);
    }
    int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { sm[w][0] = a; sm[w][1] = c; sm[w][2] = d; }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = c = d = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { a += sm[q][0]; c += sm[q][1]; d += sm[q][2]; }
    }
}

// Block-wide sum of three 64-bit integers; exact, result valid in thread 0.
__device__ __forceinline__ void block_sum3_ll(long long &a, long long &c, long long &d, long long (*sm)[3])
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
        d += __shfl_down_sync(0xffffffffu, d, o);
    }
    int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { sm[w][0] = a; sm[w][1] = c; sm[w][2] = d; }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = c = d = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { a += sm[q][0]; c += sm[q][1]; d += sm[q][2]; }
    }
}

// FP32 path: adds the block's energy sums (twice U, K and W in units of
// 2^-22) to its replica's totals.  They are exact 64-bit integer sums, so the
// order in which blocks add them does not change the result.  Called by every
// thread of the block; the sums are zero afterwards.
__device__ __forceinline__ void flush_energy(const Bufs &b, int r, long long &u, long long &k, long long &w,
                                             long long (*sm)[3])
{
    block_sum3_ll(u, k, w, sm);
    if (threadIdx.x == 0) {
        unsigned long long *e = reinterpret_cast<unsigned long long *>(b.eacc + 4 * r);
        if (u) atomicAdd(e + 0, (unsigned long long)u);
        if (k) atomicAdd(e + 1, (unsigned long long)k);
        if (w) atomicAdd(e + 2, (unsigned long long)w);
    }
    u = k = w = 0;
    __syncthreads();   // sm is written again by the next flush
}

// Last block: per-replica totals.  `fixed` (the FP32 path): the per-replica
// 64-bit integer sums that the blocks added, read and cleared for the next
// launch.  Otherwise (FP64) the per-tile partials, summed in tile order.
__device__ void reduce_partials(const Bufs &b, double *thermo, bool fixed)
{
    if (fixed) {
        for (int r = threadIdx.x; r < b.nrep; r += blockDim.x) {
            unsigned long long *e = reinterpret_cast<unsigned long long *>(b.eacc + 4 * r);
            const long long la = (long long)atomicExch(e + 0, 0ull);
            const long long lc = (long long)atomicExch(e + 1, 0ull);
            const long long ld = (long long)atomicExch(e + 2, 0ull);
            if (thermo) {
                constexpr double half_unit = 0.5 / 4194304.0;
                thermo[3 * r + 0] = half_unit * ll_to_double(la);
                thermo[3 * r + 1] = half_unit * ll_to_double(lc);
                thermo[3 * r + 2] = half_unit * ll_to_double(ld);
            }
        }
        return;
    }
    __shared__ double red[kBlock][3];
    for (int r = 0; r < b.nrep; ++r) {
        double a = 0, c = 0, d = 0;
        for (int q = b.rep_tile[r] + threadIdx.x; q < b.rep_tile[r + 1]; q += blockDim.x) {
            a += b.partial[4 * q + 0];
            c += b.partial[4 * q + 1];
            d += b.partial[4 * q + 2];
        }
        red[threadIdx.x][0] = a; red[threadIdx.x][1] = c; red[threadIdx.x][2] = d;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) {
                red[threadIdx.x][0] += red[threadIdx.x + s][0];
                red[threadIdx.x][1] += red[threadIdx.x + s][1];
                red[threadIdx.x][2] += red[threadIdx.x + s][2];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0 && thermo) {
            thermo[3 * r + 0] = red[0][0];
            thermo[3 * r + 1] = red[0][1];
            thermo[3 * r + 2] = red[0][2];
        }
        __syncthreads();
    }
}

// Drift update shared by the fused and kick-drift kernels: x += dt v, wrap
// into [0, L) (only when the fixed-point image leaves [0, 2^32)), fixed-point
// copy, and squared displacement since the last list build relative to the
// replica's threshold.
__device__ __forceinline__ float drift(const Bufs &b, const Replica &R, long long i, int nxt, unsigned id,
                                       const double xi[3], const double v[3])
{
    unsigned q[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double y = xi[k] + b.dt * v[k];
        long long qq = fix_round(y, R.to_q[k]);
        if ((unsigned long long)qq >= 4294967296ULL) {
            y = wrap1(y, R.L[k]);
            qq = fix_round(y, R.to_q[k]);
        }
        b.x[nxt][k * b.S + i] = y;
        b.v[nxt][k * b.S + i] = v[k];
        q[k] = (unsigned)(qq & 0xffffffffLL);
    }
    uint4 p = make_uint4(q[0], q[1], q[2], id);
    b.pos[nxt][i] = p;
    uint4 r = b.xref[i];
    float dx = (float)(int)(p.x - r.x) * R.qs[0];
    float dy = (float)(int)(p.y - r.y) * R.qs[1];
    float dz = (float)(int)(p.z - r.z) * R.qs[2];
    return (dx * dx + dy * dy + dz * dz) / R.disp2_thr;
}

// Block-wide maximum of a float; result valid in thread 0.
__device__ __forceinline__ float block_max(float v, float *sm)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) v = fmaxf(v, sm[q]);
    return v;
}

// End-of-kernel bookkeeping by the last block to finish: energy totals, the
// work counter, and for kernels that drifted the buffer flip, the step
// counter and the rebuild decision for the next step.
__device__ void finish(const Bufs &b, bool drifted, bool energy, bool tiled, float ratio_blk, bool fixed = false)
{
    if (!drifted && !energy && !tiled) return;
    __shared__ bool last;
    if (threadIdx.x == 0) {
        if (drifted && ratio_blk > 0.0f) atomicMax(&b.ctl->disp2_bits, __float_as_uint(ratio_blk));
        __threadfence();
        unsigned prev = atomicAdd(&b.ctl->done_force, 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (energy) {
        // a graph-launched md_step records every step into its ring slot
        double *out = b.thermo;
        if (!out && b.thermo_ring) out = b.thermo_ring + 3 * (long long)b.nrep * b.ctl->rec;
        reduce_partials(b, out, fixed);
        if (!b.thermo && b.thermo_ring && threadIdx.x == 0) b.ctl->rec += 1;
    }
    if (threadIdx.x == 0) {
        if (drifted) {
            unsigned bits = atomicExch(&b.ctl->disp2_bits, 0u);
            b.ctl->rebuild = (__uint_as_float(bits) > 1.0f) ? 1 : 0;
            b.ctl->cur ^= 1;
            b.ctl->step += 1;
            if (b.g_while) {                    // inside the graph's step loop
                const long long left = b.ctl->steps_left - 1;
                b.ctl->steps_left = left;
                // every block has added its error bits before counting itself
                // done, so an error latched by this launch ends the loop now
                const int e = *(volatile int *)&b.ctl->err;
                cudaGraphSetConditional(b.g_while, (left > 0 && e == 0) ? 1u : 0u);
            }
        }
        if (tiled) b.ctl->tile_next = 0u;
        b.ctl->done_force = 0u;
    }
}

// FP32 pair terms of one neighbour: LJ force scalar masked to zero unless
// `in`, and the fixed-point accumulation of force, energy and virial.
struct Acc32 {
    unsigned hx, lx, hy, ly, hz, lz;
    // energies: sums over the interacting pairs of s6 = (sigma/r)^6 and of
    // g = s6 (2 s6 - 1), and their count.  s6 (s6 - 1) = (g - s6) / 2, so the
    // pair energy is 2 eps (sg - s6) - n V(r_cut) and the virial 24 eps sg.
    // Two partial sums each (the lanes of the packed loop), added at the end;
    // the packed loop counts in FP32 as r^2 times its masked 1/r^2 (1 to
    // rounding per interacting pair, 0 otherwise), the single-pair path in nin.
    float2 s6, sg, cnt;
    int nin;
};

// The shifted LJ energy summed over the pairs of these sums: 4 eps times the
// sum of s6 (s6 - 1), minus V(r_cut) per interacting pair (FP32).
__device__ __forceinline__ float pair_energy(const Replica &R, const Acc32 &a)
{
    return R.eps4_f * 0.5f * ((a.sg.x + a.sg.y) - (a.s6.x + a.s6.y)) - R.vshift_f * ((a.cnt.x + a.cnt.y) + (float)a.nin);
}

// slot of halo index h (pieces are in ascending halo order)
__device__ __forceinline__ int halo_slot(const Piece *pc, int np, int h)
{
    int q = 0;
    while (q + 1 < np && h >= pc[q + 1].hoff) ++q;
    return pc[q].slot0 + (h - pc[q].hoff);
}

// bounds checks of the checked build (md_ok): a list entry within the
// staged halo of hsize entries (else entry 0), a slot within the S slots
// (else slot i, the particle's own)
__device__ __forceinline__ int checked_entry(Ctl *ctl, int h, int hsize, int site)
{
    return md_ok(ctl, (unsigned)h < (unsigned)hsize, site, h) ? h : 0;
}

__device__ __forceinline__ long long checked_slot(Ctl *ctl, long long j, long long S, long long i,
                                                  int site = kSiteForceSlot)
{
    return md_ok(ctl, j >= 0 && j < S, site, j) ? j : i;
}

// All lengths in fixed-point units u of the x axis: r2 and d in u, the force
// scalar fs in force / u (constants pre-scaled), so fs * d is the force.
template <bool ENERGY>
__device__ __forceinline__ void pair32(float dx, float dy, float dz, float r2, bool in, float sig2, float eps24,
                                       Acc32 &a)
{
    const float ir2 = rcp_approx(r2);
    const float s2 = sig2 * ir2;
    const float s6 = s2 * s2 * s2;
    const float g = s6 * (2.0f * s6 - 1.0f);
    const float fs = in ? eps24 * g * ir2 : 0.0f;
    fx_acc2(fs, dx, a.hx, a.lx);
    fx_acc2(fs, dy, a.hy, a.ly);
    fx_acc2(fs, dz, a.hz, a.lz);
    if (ENERGY) {
        a.s6.x += in ? s6 : 0.0f;
        a.sg.x += in ? g : 0.0f;
        a.nin += in ? 1 : 0;
    }
}

// pair32 for two neighbours (the same arithmetic, packed); the fixed-point
// pieces carry the bias of fx_acc2x2
template <bool ENERGY>
__device__ __forceinline__ void pair32x2(float2 dx, float2 dy, float2 dz, float2 r2, bool in0, bool in1, float sig2,
                                         float eps24, Acc32 &a)
{
    // 1/r^2 masked to 0 outside the cutoff (and for the r = 0 padding), so
    // that s6, g, the force scalar and the energy terms all vanish there
    float2 ir2 = make_float2(rcp_approx(r2.x), rcp_approx(r2.y));
    ir2.x = in0 ? ir2.x : 0.0f;
    ir2.y = in1 ? ir2.y : 0.0f;
    const float2 s2 = __fmul2_rn(make_float2(sig2, sig2), ir2);
    const float2 s6 = __fmul2_rn(__fmul2_rn(s2, s2), s2);
    const float2 g = __fmul2_rn(s6, __ffma2_rn(make_float2(2.0f, 2.0f), s6, make_float2(-1.0f, -1.0f)));
    const float2 fs = __fmul2_rn(__fmul2_rn(make_float2(eps24, eps24), g), ir2);
    fx_acc2x2(fs, dx, a.hx, a.lx);
    fx_acc2x2(fs, dy, a.hy, a.ly);
    fx_acc2x2(fs, dz, a.hz, a.lz);
    if (ENERGY) {
        a.s6 = __fadd2_rn(a.s6, s6);
        a.sg = __fadd2_rn(a.sg, g);
        a.cnt = __ffma2_rn(ir2, r2, a.cnt);
    }
}

// separation of two fixed-point positions in units u of the x axis
template <bool CUBIC>
__device__ __forceinline__ void sep_u(uint4 a, uint4 c, float ry, float rz, float &dx, float &dy, float &dz, float &r2)
{
    dx = (float)(int)(a.x - c.x);
    dy = (float)(int)(a.y - c.y);
    dz = (float)(int)(a.z - c.z);
    if (!CUBIC) { dy *= ry; dz *= rz; }
    // the rounding order of the packed loop, so that both see the same r^2
    r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// FP32 neighbour loop of one particle: padded list, branch-free arithmetic;
// pairs within rounding of r_cut are settled afterwards in FP64.
template <bool ENERGY, bool CUBIC, bool LSMEM>
__device__ __forceinline__ void neighbours32(const Replica &R, const uint4 *hpos, const unsigned short *nb, int Pt,
                                             int n, int npad, uint4 pi, const double *X, long long S, long long i,
                                             const Piece *pc, int np, Acc32 &a, int &err, Ctl *ctl, int hsize)
{
    const float ry = R.ry, rz = R.rz;
    const float lo = R.rc2_lo_u, hi = R.rc2_hi_u, fmax2 = R.fmax2_u;
    const float sig2 = R.sig2_u, eps24 = R.eps24_u;
    // a pair within rounding of r_cut, or closer than the fixed-point range
    // allows: both rare, so one flag, and the pass below tells them apart
    bool rare = false;
    for (int k0 = 0; k0 < npad; k0 += kU) {
        int hh[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u)
            hh[u] = checked_entry(ctl, LSMEM ? nb[(k0 + u) * Pt] : __ldg(nb + (long long)(k0 + u) * Pt), hsize,
                                  kSiteForceHalo);
#pragma unroll
        for (int u = 0; u < kU; u += 2) {
            const uint4 q0 = lds128(hpos + hh[u]), q1 = lds128(hpos + hh[u + 1]);
            float2 dx = make_float2((float)(int)(pi.x - q0.x), (float)(int)(pi.x - q1.x));
            float2 dy = make_float2((float)(int)(pi.y - q0.y), (float)(int)(pi.y - q1.y));
            float2 dz = make_float2((float)(int)(pi.z - q0.z), (float)(int)(pi.z - q1.z));
            if (!CUBIC) {
                dy = __fmul2_rn(dy, make_float2(ry, ry));
                dz = __fmul2_rn(dz, make_float2(rz, rz));
            }
            const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
            // padding entries are the particle itself (r^2 = 0)
            const bool nz0 = r2.x > 0.0f, nz1 = r2.y > 0.0f;
            const bool in0 = (r2.x < lo) & nz0, in1 = (r2.y < lo) & nz1;
            rare |= ((r2.x < hi) & !(r2.x < lo)) | ((r2.y < hi) & !(r2.y < lo)) | ((r2.x < fmax2) & nz0) |
                    ((r2.y < fmax2) & nz1);
            pair32x2<ENERGY>(dx, dy, dz, r2, in0, in1, sig2, eps24, a);
        }
    }
    {
        // remove the bias of the npad packed terms of every accumulator
        const unsigned bias = (unsigned)npad * kMagicBits;
        a.hx -= bias; a.lx -= bias; a.hy -= bias; a.ly -= bias; a.hz -= bias; a.lz -= bias;
    }
    if (rare) {
        // pairs within rounding of r_cut: membership decided in FP64 from the
        // master positions, as in the FP64 reference; and pairs too close for
        // the fixed-point sums
        bool tooclose = false;
        for (int k = 0; k < n; ++k) {
            const int h = checked_entry(ctl, nb[(long long)k * Pt], hsize, kSiteForceHalo);
            float dx, dy, dz, r2;
            sep_u<CUBIC>(pi, hpos[h], ry, rz, dx, dy, dz, r2);
            tooclose |= (r2 < fmax2) & (r2 > 0.0f);
            if (!(r2 < lo) && r2 < hi && r2_exact(X, S, i, checked_slot(ctl, halo_slot(pc, np, h), S, i), R.L) < R.rc2)
                pair32<ENERGY>(dx, dy, dz, r2, true, sig2, eps24, a);
        }
        if (tooclose) err |= kErrFixed;
    }
}

// ---------------------------------------------------------------- half list
// Newton's third law (Sec. 2.1.2): a half list holds each pair once, and the
// pair force goes to both particles.  The two exactly rounded pieces of each
// component are those of fx_acc2 / fx_acc2x2, so round(f_ij 2^22) is the
// same integer whichever end evaluates the pair, and its negation is
// round(f_ji 2^22) (the rounding is odd): the half-list forces are the
// full-list forces bit for bit.

// round(a c 2^22) of one lane as a 64-bit fixed-point value, from the biased
// pieces t1 = kMagic + round(a c), t2 = kMagic + round(r 2^22)
__device__ __forceinline__ long long fx_value(float t1, float t2)
{
    return (long long)(int)(__float_as_uint(t1) - kMagicBits) * 4194304LL +
           (long long)(int)(__float_as_uint(t2) - kMagicBits);
}

// fx_acc2x2 that also returns both lanes' values
__device__ __forceinline__ void fx_acc2x2_v(float2 a, float2 c, unsigned &hi, unsigned &lo, long long &v0,
                                            long long &v1)
{
    const float2 M = make_float2(kMagic, kMagic);
    const float2 t1 = __ffma2_rn(a, c, M);
    const float2 nh = __ffma2_rn(t1, make_float2(-1.0f, -1.0f), M);
    const float2 r = __ffma2_rn(a, c, nh);
    const float2 t2 = __ffma2_rn(r, make_float2(kFixScale, kFixScale), M);
    hi += __float_as_uint(t1.x) + __float_as_uint(t1.y);
    lo += __float_as_uint(t2.x) + __float_as_uint(t2.y);
    v0 = fx_value(t1.x, t2.x);
    v1 = fx_value(t1.y, t2.y);
}

// the scalar value of fx_acc2 (same instructions, same rounding)
__device__ __forceinline__ long long fx_value1(float a, float c)
{
    const float t1 = __fmaf_rn(a, c, kMagic);
    const float h = __fsub_rn(t1, kMagic);
    const float r = __fmaf_rn(a, c, -h);
    const float t2 = __fmaf_rn(r, kFixScale, kMagic);
    return fx_value(t1, t2);
}

// subtract v from the fixed-point sum at *p (the reaction on the partner)
__device__ __forceinline__ void red_sub(long long *p, long long v)
{
    atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)(-v));
}

// pair32x2 for the half list: the same arithmetic, plus the reactions of
// both neighbours (slots s0, s1) into the global fixed-point sums
template <bool ENERGY>
__device__ __forceinline__ void pair32x2_half(float2 dx, float2 dy, float2 dz, float2 r2, bool in0, bool in1,
                                              float sig2, float eps24, Acc32 &a, long long *Fq, long long S,
                                              unsigned s0, unsigned s1)
{
    // 1/r^2 masked to 0 outside the cutoff (and for the r = 0 padding), so
    // that s6, g, the force scalar and the energy terms all vanish there
    float2 ir2 = make_float2(rcp_approx(r2.x), rcp_approx(r2.y));
    ir2.x = in0 ? ir2.x : 0.0f;
    ir2.y = in1 ? ir2.y : 0.0f;
    const float2 s2 = __fmul2_rn(make_float2(sig2, sig2), ir2);
    const float2 s6 = __fmul2_rn(__fmul2_rn(s2, s2), s2);
    const float2 g = __fmul2_rn(s6, __ffma2_rn(make_float2(2.0f, 2.0f), s6, make_float2(-1.0f, -1.0f)));
    const float2 fs = __fmul2_rn(__fmul2_rn(make_float2(eps24, eps24), g), ir2);
    long long x0, x1, y0, y1, z0, z1;
    fx_acc2x2_v(fs, dx, a.hx, a.lx, x0, x1);
    fx_acc2x2_v(fs, dy, a.hy, a.ly, y0, y1);
    fx_acc2x2_v(fs, dz, a.hz, a.lz, z0, z1);
    if (in0) { red_sub(Fq + s0, x0); red_sub(Fq + S + s0, y0); red_sub(Fq + 2 * S + s0, z0); }
    if (in1) { red_sub(Fq + s1, x1); red_sub(Fq + S + s1, y1); red_sub(Fq + 2 * S + s1, z1); }
    if (ENERGY) {
        a.s6 = __fadd2_rn(a.s6, s6);
        a.sg = __fadd2_rn(a.sg, g);
        a.cnt = __ffma2_rn(ir2, r2, a.cnt);
    }
}

// neighbours32 over a half list: the staged halo carries each particle's slot
// in .w, where the reactions go
template <bool ENERGY, bool CUBIC>
__device__ __forceinline__ void neighbours32_half(const Replica &R, const uint4 *hpos, const unsigned short *nb, int Pt,
                                                  int n, int npad, uint4 pi, const double *X, long long S, long long i,
                                                  const Piece *pc, int np, Acc32 &a, int &err, long long *Fq,
                                                  Ctl *ctl, int hsize)
{
    const float ry = R.ry, rz = R.rz;
    const float lo = R.rc2_lo_u, hi = R.rc2_hi_u, fmax2 = R.fmax2_u;
    const float sig2 = R.sig2_u, eps24 = R.eps24_u;
    // a pair within rounding of r_cut, or closer than the fixed-point range
    // allows: both rare, so one flag, and the pass below tells them apart
    bool rare = false;
    for (int k0 = 0; k0 < npad; k0 += kU) {
        int hh[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) hh[u] = checked_entry(ctl, nb[(k0 + u) * Pt], hsize, kSiteForceHalo);
#pragma unroll
        for (int u = 0; u < kU; u += 2) {
            uint4 q0 = hpos[hh[u]], q1 = hpos[hh[u + 1]];
            q0.w = (unsigned)checked_slot(ctl, (int)q0.w, S, i);   // where the reactions go
            q1.w = (unsigned)checked_slot(ctl, (int)q1.w, S, i);
            float2 dx = make_float2((float)(int)(pi.x - q0.x), (float)(int)(pi.x - q1.x));
            float2 dy = make_float2((float)(int)(pi.y - q0.y), (float)(int)(pi.y - q1.y));
            float2 dz = make_float2((float)(int)(pi.z - q0.z), (float)(int)(pi.z - q1.z));
            if (!CUBIC) {
                dy = __fmul2_rn(dy, make_float2(ry, ry));
                dz = __fmul2_rn(dz, make_float2(rz, rz));
            }
            const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
            const bool nz0 = r2.x > 0.0f, nz1 = r2.y > 0.0f;
            const bool in0 = (r2.x < lo) & nz0, in1 = (r2.y < lo) & nz1;
            rare |= ((r2.x < hi) & !(r2.x < lo)) | ((r2.y < hi) & !(r2.y < lo)) | ((r2.x < fmax2) & nz0) |
                    ((r2.y < fmax2) & nz1);
            pair32x2_half<ENERGY>(dx, dy, dz, r2, in0, in1, sig2, eps24, a, Fq, S, q0.w, q1.w);
        }
    }
    {
        const unsigned bias = (unsigned)npad * kMagicBits;
        a.hx -= bias; a.lx -= bias; a.hy -= bias; a.ly -= bias; a.hz -= bias; a.lz -= bias;
    }
    if (rare) {
        bool tooclose = false;
        for (int k = 0; k < n; ++k) {
            const int h = checked_entry(ctl, nb[k * Pt], hsize, kSiteForceHalo);
            uint4 q = hpos[h];
            q.w = (unsigned)checked_slot(ctl, (int)q.w, S, i);
            float dx, dy, dz, r2;
            sep_u<CUBIC>(pi, q, ry, rz, dx, dy, dz, r2);
            tooclose |= (r2 < fmax2) & (r2 > 0.0f);
            if (!(r2 < lo) && r2 < hi && r2_exact(X, S, i, (long long)q.w, R.L) < R.rc2) {
                pair32<ENERGY>(dx, dy, dz, r2, true, sig2, eps24, a);
                // the force scalar of pair32, for the partner's share
                const float ir2 = rcp_approx(r2);
                const float s2 = sig2 * ir2;
                const float s6 = s2 * s2 * s2;
                const float fs = eps24 * (s6 * (2.0f * s6 - 1.0f)) * ir2;
                red_sub(Fq + q.w, fx_value1(fs, dx));
                red_sub(Fq + S + q.w, fx_value1(fs, dy));
                red_sub(Fq + 2 * S + q.w, fx_value1(fs, dz));
            }
        }
        if (tooclose) err |= kErrFixed;
    }
}

// Cosine angle term K (1 - cos theta) of a triple (a, b, c) with bond vectors
// b1 = x_b - x_a, b2 = x_c - x_b and c = b1.b2 / (|b1| |b2|): the force on the
// particle of the given role, F_a = -K (b2/(l1 l2) - c b1/l1^2),
// F_c = K (b1/(l1 l2) - c b2/l2^2), F_b = -(F_a + F_c); and the energy.
template <class Real>
__device__ __forceinline__ void angle_term(const Real b1[3], const Real b2[3], Real K, Real fa[3], Real fc[3], Real &u)
{
    const Real l1s = b1[0] * b1[0] + b1[1] * b1[1] + b1[2] * b1[2];
    const Real l2s = b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2];
    const Real l12 = sqrt(l1s) * sqrt(l2s);
    const Real c = (b1[0] * b2[0] + b1[1] * b2[1] + b1[2] * b2[2]) / l12;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        fa[k] = -K * (b2[k] / l12 - c * b1[k] / l1s);
        fc[k] = K * (b1[k] / l12 - c * b2[k] / l2s);
    }
    u = K * (Real(1) - c);
}


// a4 + a5: forces on every particle of a tile from its Verlet list, with
// the neighbour positions read from the tile's halo in shared memory, then
// the velocity-Verlet update of that particle.  Persistent blocks take tiles
// from a work counter; the first warp stages each FP32 tile by bulk (TMA)
// copies (issue_tile_bulk).
// HALF (FP32 only): the second kernel of a half-list step.  k_pairs_half has
// left each particle's total pair force in the fixed-point sums Fq; this pass
// takes it from there (and clears it) instead of walking a list, then does
// exactly what the full-list kernel does with the force.
template <int PREC, int MODE, bool ENERGY, bool HALF = false>
__global__ void __launch_bounds__(kBlock, PREC == 1 ? MDK_FORCE_MIN_BLOCKS : 1) k_force(Bufs b)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // tile records and halo pieces, double-buffered: the next tile's are
    // copied in by one warp while this one is computed
    __shared__ Piece pcb[2][kMaxPieces + 1];
    __shared__ Tile tlb[2];
    __shared__ int s_npb[2];
    __shared__ int s_tile, s_self, s_next, s_issued;
    __shared__ int s_nn[kTileMax];
    __shared__ double sm3[kBlock / 32][3];
    __shared__ long long sml[kBlock / 32][3];
    __shared__ float smr[kBlock / 32];
    __shared__ __align__(8) unsigned long long s_mbar;   // completion of a tile's bulk copies
    __shared__ __align__(8) unsigned long long s_p1bar;  // every thread past its pair sums
    if (block_uniform(b.ctl->err != 0)) {
        // inside a graph-launched step loop nothing else would clear the
        // loop's condition: a latched error ends the loop here
        if (b.g_while && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(b.g_while, 0u);
        return;
    }
    // FP32 full-list tiles are staged by bulk (TMA) copies: thread 0 arms the
    // barrier and copies the halo pieces and the list block, all threads wait
    constexpr bool kBulk = (PREC == 1 && !HALF);
    unsigned phase = 0;
    unsigned p1phase = 0;
    if (kBulk && threadIdx.x == 0) {
        mbar_init(&s_mbar, 1);
        mbar_init(&s_p1bar, blockDim.x);
    }
    const int cur = b.ctl->cur, nxt = cur ^ 1;
    const long long step = b.ctl->step;
    const double *X = b.x[cur];
    const uint4 *P = b.pos[cur];
    uint4 *hpos = reinterpret_cast<uint4 *>(smem_raw);
    double *hx = reinterpret_cast<double *>(smem_raw);
    double *hy = hx + b.hcap, *hz = hy + b.hcap;
    unsigned short *lst = reinterpret_cast<unsigned short *>(smem_raw + (size_t)b.hcap * (PREC == 1 ? sizeof(uint4) : 3 * sizeof(double)));
    float ratio = 0.0f;
    int err = 0;
    int buf = 0;           // which tile buffer holds tile t
    bool have = false;     // whether it was prefetched
    // FP32 path: energies as integers, twice the energy in units of 2^-22,
    // summed over this block's tiles until the replica changes
    long long uf = 0, wf = 0, kf = 0;
    int rcur = -1;
    if (threadIdx.x == 0) {
        s_tile = (int)atomicAdd(&b.ctl->tile_next, 1u);
        s_issued = 0;
    }
    __syncthreads();
    for (;;) {
        const int t = s_tile;
        const bool issued = s_issued != 0;   // this tile's copies went out during the last one
        __syncthreads();
        if (t >= b.ctl->ntiles) break;
        // the next tile is claimed now and published at the end of this one
        int t_next = 0;
        if (threadIdx.x == 0) t_next = (int)atomicAdd(&b.ctl->tile_next, 1u);
        if (!have) load_tile(b, t, tlb[buf], pcb[buf], s_npb[buf]);
        __syncthreads();
        Piece *const pc = pcb[buf];
        const Tile &tl = tlb[buf];
        const Replica &R = b.rep[tl.rep];
        const int np = s_npb[buf];
        const int Pt = tl.s1 - tl.s0;
        if (ENERGY && PREC == 1 && tl.rep != rcur) {   // block-uniform
            if (rcur >= 0) flush_energy(b, rcur, uf, kf, wf, sml);
            rcur = tl.rep;
        }
        if (!HALF && pc[np].hoff > b.hcap) {          // the list build rejects such tiles first
            err |= kErrList;
            if (threadIdx.x == 0) { s_tile = t_next; s_issued = 0; }
            __syncthreads();
            have = false;
            continue;
        }
        const bool own_staged = Pt <= kTileMax;
        if (!HALF) {   // halo and list block (the half-list pass reads no list)
            if (own_staged)
                for (int p = threadIdx.x; p < Pt; p += blockDim.x) cp_async4(&s_nn[p], &b.nn[tl.s0 + p]);
            if (threadIdx.x == 0) s_self = tile_self_offset(R, tl, pc, np);
            if (kBulk) {
                if (threadIdx.x < 32 && !issued) issue_tile_bulk(b, tl, pc, np, P, hpos, lst, &s_mbar, threadIdx.x);
            } else if (PREC == 1) stage_halo<uint4>(pc, np, [&](int h, int j) { cp_async16(&hpos[h], &P[j]); });
            else stage_halo<double>(pc, np, [&](int h, int j) {
                cp_async8(&hx[h], &X[j]);
                cp_async8(&hy[h], &X[b.S + j]);
                cp_async8(&hz[h], &X[2 * b.S + j]);
            });
            // the tile's lists: kmax rows of Pt entries, one contiguous block
            if (!kBulk && tl.kmax * Pt <= kListStage * kTileMax) {
                const unsigned short *src = b.nbr + nbr_index(tl.s0, Pt, b.K, 0, 0);
                const int total = tl.kmax * Pt;            // entries; the block starts 64-byte aligned
                const int nvec = total >> 3;
                const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
                uint4 *d4 = reinterpret_cast<uint4 *>(lst);
                for (int m = threadIdx.x; m < nvec; m += blockDim.x) cp_async16(d4 + m, s4 + m);
                for (int m = (nvec << 3) + threadIdx.x; m < total; m += blockDim.x) lst[m] = src[m];
            }
            cp_async_wait_all();
        }
        if (threadIdx.x == 0) s_next = t_next;
        bool late = false;
        if (kBulk) {
            late = !mbar_wait(&s_mbar, phase);
            phase ^= 1u;
        }
        if (__syncthreads_or(late)) {   // a bulk copy never completed: stop, report
            err |= kErrTimeout;
            break;
        }
        // FP64: the staged halo moved into the tile's periodic frame (each
        // coordinate within half a box of the tile centre; the tile's own
        // particles are halo entries too).  With at least 3 cells per axis and a
        // tile at least 3 cells narrower than its row, every pair closer than a
        // cell edge then has its minimum-image separation as the plain
        // difference, so the neighbour loop takes no minimum image; any farther
        // pair is beyond r_cut in every image.
        const bool shifted = PREC == 0 && R.ncell[1] >= 3 && R.ncell[2] >= 3 && tl.x1 - tl.x0 <= R.ncell[0] - 3;
        if (shifted) {
            const double c0 = 0.5 * (tl.x0 + tl.x1) * R.L[0] / R.ncell[0];
            const double c1 = (tl.cy + 0.5) * R.L[1] / R.ncell[1];
            const double c2 = (tl.cz + 0.5) * R.L[2] / R.ncell[2];
            const double g0 = 0.5 * R.L[0], g1 = 0.5 * R.L[1], g2 = 0.5 * R.L[2];
            for (int h = threadIdx.x; h < pc[np].hoff; h += blockDim.x) {
                const double t0 = hx[h] - c0, t1 = hy[h] - c1, t2 = hz[h] - c2;
                if (t0 > g0) hx[h] -= R.L[0]; else if (t0 < -g0) hx[h] += R.L[0];
                if (t1 > g1) hy[h] -= R.L[1]; else if (t1 < -g1) hy[h] += R.L[1];
                if (t2 > g2) hz[h] -= R.L[2]; else if (t2 < -g2) hz[h] += R.L[2];
            }
            __syncthreads();
        }
        // the last warp copies the next tile's record and pieces into the other
        // buffer while the tile is computed (not in the half-list pass, which
        // stages nothing and has little work per tile to hide the copy behind)
        const int tn = s_next;
        const bool pref = !HALF && tn < b.ctl->ntiles;
        if (pref && threadIdx.x >= blockDim.x - 32)
            prefetch_tile_async(b, tn, tlb[buf ^ 1], pcb[buf ^ 1], s_npb[buf ^ 1], threadIdx.x & 31);
        const bool lstaged = tl.kmax * Pt <= kListStage * kTileMax;
        double ui = 0.0, wi = 0.0, ki = 0.0;
        // Per particle: the pair sums (phase 1, which reads the staged halo
        // and list) and everything after them (phase 2: bonded terms, Langevin
        // force, integration, energies), which reads neither.
        struct PState {
            uint4 pi;
            double Fd[3];
            double fscale, ckick;
        };
        auto phase1 = [&](long long i, PState &ps) {
            if (MODE == kModeFused) {
                // this particle's integration state, needed after the pair loop
                prefetch_l1(&b.v[cur][i]); prefetch_l1(&b.v[cur][b.S + i]); prefetch_l1(&b.v[cur][2 * b.S + i]);
                prefetch_l1(&X[i]); prefetch_l1(&X[b.S + i]); prefetch_l1(&X[2 * b.S + i]);
                prefetch_l1(&b.xref[i]);
            }
            ps.pi = (PREC == 1 && !HALF) ? hpos[checked_entry(b.ctl, s_self + (int)(i - tl.s0), pc[np].hoff, kSiteForceOwn)]
                                         : P[i];
            const uint4 pi = ps.pi;
            const int n = min(own_staged ? s_nn[i - tl.s0] : b.nn[i], b.K);
            const int npad = min(((n + kPad - 1) / kPad) * kPad, b.K);
            const unsigned short *nb = b.nbr + nbr_index(tl.s0, Pt, b.K, 0, (int)(i - tl.s0));   // entry k at nb[k Pt]
            double *Fd = ps.Fd;
            Fd[0] = Fd[1] = Fd[2] = 0.0;
            double &fscale = ps.fscale;
            fscale = 1.0;
            double &ckick = ps.ckick;
            ckick = b.half_dt_over_m;            // half kick per unit of Fd
            if (PREC == 1 && HALF) {
                // the pair sums of k_pairs_half, cleared for the next step
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    Fd[k] = ll_to_double(b.Fq[k * b.S + i]);
                    b.Fq[k * b.S + i] = 0;
                }
                fscale = kFixInv;
                ckick = b.half_dt_over_m_fix;
            } else if (PREC == 1) {
                Acc32 a = {0u, 0u, 0u, 0u, 0u, 0u, make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f), 0};
                if (lstaged) {
                    const unsigned short *nbs = lst + (i - tl.s0);
                    if (R.cubic) neighbours32<ENERGY, true, true>(R, hpos, nbs, Pt, n, npad, pi, X, b.S, i, pc, np, a, err, b.ctl, pc[np].hoff);
                    else neighbours32<ENERGY, false, true>(R, hpos, nbs, Pt, n, npad, pi, X, b.S, i, pc, np, a, err, b.ctl, pc[np].hoff);
                } else {
                    if (R.cubic) neighbours32<ENERGY, true, false>(R, hpos, nb, Pt, n, npad, pi, X, b.S, i, pc, np, a, err, b.ctl, pc[np].hoff);
                    else neighbours32<ENERGY, false, false>(R, hpos, nb, Pt, n, npad, pi, X, b.S, i, pc, np, a, err, b.ctl, pc[np].hoff);
                }
                const unsigned hs[3] = {a.hx, a.hy, a.hz}, ls[3] = {a.lx, a.ly, a.lz};
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    Fd[k] = ll_to_double((long long)(int)hs[k] * 4194304LL + (long long)(int)ls[k]);
                fscale = kFixInv;
                ckick = b.half_dt_over_m_fix;
                if (ENERGY) {
                    // twice this particle's pair energy and virial, in FP32, to fixed point
                    uf += fx_round(pair_energy(R, a));
                    wf += fx_round(R.eps24_f * (a.sg.x + a.sg.y));
                }
            } else {
                // in the tile's frame the particle's own coordinates come from its
                // (shifted) halo entry: a particle that crossed the periodic
                // boundary since the last build keeps its cell but wrapped
                const int own = checked_entry(b.ctl, s_self + (int)(i - tl.s0), pc[np].hoff, kSiteForceOwn);
                const double xi0 = shifted ? hx[own] : X[i], xi1 = shifted ? hy[own] : X[b.S + i],
                             xi2 = shifted ? hz[own] : X[2 * b.S + i];
                const double L0 = R.L[0], L1 = R.L[1], L2 = R.L[2];
                const double h0 = 0.5 * L0, h1 = 0.5 * L1, h2 = 0.5 * L2;
                const double eps24 = 24.0 * R.eps, eps4 = 4.0 * R.eps, sig2 = R.sigma * R.sigma;
                const double rc2 = R.rc2, vsh = R.vshift;
                const double band = 1e-12 * rc2;
                const unsigned short *nbs = lst + (i - tl.s0);
                for (int k = 0; k < n; ++k) {
                    const int h = checked_entry(b.ctl, lstaged ? nbs[k * Pt] : __ldg(nb + (long long)k * Pt),
                                                pc[np].hoff, kSiteForceHalo);
                    double dx = xi0 - hx[h], dy = xi1 - hy[h], dz = xi2 - hz[h];
                    if (!shifted) {
                        dx = dx > h0 ? dx - L0 : (dx < -h0 ? dx + L0 : dx);
                        dy = dy > h1 ? dy - L1 : (dy < -h1 ? dy + L1 : dy);
                        dz = dz > h2 ? dz - L2 : (dz < -h2 ? dz + L2 : dz);
                    }
                    const double r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 < rc2 + band) {
                        bool in = r2 < rc2 - band;
                        if (!in) in = r2_exact(X, b.S, i, checked_slot(b.ctl, halo_slot(pc, np, h), b.S, i), R.L) < rc2;
                        if (in && R.soft) {
                            // cosine push-off A (1 + cos(pi r / r_cut)), A = eps:
                            // -dV/dr = (pi A / r_cut) sin(pi r / r_cut), none at r = 0
                            const double r = sqrt(r2);
                            double sn, cs;
                            sincospi(r / R.rc, &sn, &cs);
                            const double fs = r > 0.0 ? (CUDART_PI * R.eps / R.rc) * sn / r : 0.0;
                            Fd[0] += fs * dx;
                            Fd[1] += fs * dy;
                            Fd[2] += fs * dz;
                            if (ENERGY) {
                                ui += 0.5 * (R.eps * (1.0 + cs));
                                wi += 0.5 * fs * r2;
                            }
                        } else if (in) {
                            const double ir2 = rcp_newton(r2);
                            const double s2 = sig2 * ir2;
                            const double s6 = s2 * s2 * s2;
                            const double fs = eps24 * s6 * (2.0 * s6 - 1.0) * ir2;
                            Fd[0] += fs * dx;
                            Fd[1] += fs * dy;
                            Fd[2] += fs * dz;
                            if (ENERGY) {
                                ui += 0.5 * (eps4 * s6 * (s6 - 1.0) - vsh);
                                wi += 0.5 * fs * r2;
                            }
                        }
                    }
                }
                if (!isfinite(Fd[0]) || !isfinite(Fd[1]) || !isfinite(Fd[2])) err |= kErrNonfinite;
            }
        };
        auto phase2 = [&](long long i, PState &ps) {
            const uint4 pi = ps.pi;
            double *Fd = ps.Fd;
            double &fscale = ps.fscale;
            double &ckick = ps.ckick;
            // FENE bonds of this particle (Sec. 4), both ends of every bond
            // visited; in FP32 mode the bond force joins the fixed-point sum
            if (b.has_bonds) {
                const int id = (int)pi.w;
                for (int q = b.bond_off[id]; q < b.bond_off[id + 1]; ++q) {
                    const int sj = (int)checked_slot(b.ctl, b.bond_pslot[q], b.S, i, kSiteBondSlot);
                    if (PREC == 1) {
                        const uint4 pj = P[sj];
                        const float dx = (float)(int)(pi.x - pj.x) * R.qs[0];
                        const float dy = (float)(int)(pi.y - pj.y) * R.qs[1];
                        const float dz = (float)(int)(pi.z - pj.z) * R.qs[2];
                        const float r2 = dx * dx + dy * dy + dz * dz;
                        const float qf = 1.0f - r2 / b.fene_R02_f;
                        if (!(qf > 0.0f)) { err |= kErrBond; continue; }
                        const float c = -b.fene_K_f / qf;
                        unsigned h = 0, l = 0;
                        fx_acc2(c, dx, h, l); Fd[0] += ll_to_double((long long)(int)h * 4194304LL + (long long)(int)l); h = l = 0;
                        fx_acc2(c, dy, h, l); Fd[1] += ll_to_double((long long)(int)h * 4194304LL + (long long)(int)l); h = l = 0;
                        fx_acc2(c, dz, h, l); Fd[2] += ll_to_double((long long)(int)h * 4194304LL + (long long)(int)l);
                        if (ENERGY) {
                            uf += fix_round(-0.5 * b.fene_K * b.fene_R02 * log((double)qf), 4194304.0);
                            wf += fix_round((double)(c * r2), 4194304.0);
                        }
                    } else {
                        double d[3];
                        for (int k = 0; k < 3; ++k) {
                            double tt = X[k * b.S + i] - X[k * b.S + sj];
                            d[k] = tt - R.L[k] * rint(tt / R.L[k]);
                        }
                        const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        const double qd = 1.0 - r2 / b.fene_R02;
                        if (!(qd > 0.0)) { err |= kErrBond; continue; }
                        const double c = -b.fene_K / qd;
                        for (int k = 0; k < 3; ++k) Fd[k] += c * d[k];
                        if (ENERGY) {
                            ui += 0.5 * (-0.5 * b.fene_K * b.fene_R02 * log(qd));
                            wi += 0.5 * c * r2;
                        }
                    }
                }
            }
            // angle triples of this particle (Sec. 4), every triple visited
            // by its three particles; in FP32 mode the force joins the
            // fixed-point sum
            if (b.has_angles) {
                const int id = (int)pi.w;
                for (int q = b.ang_off[id]; q < b.ang_off[id + 1]; ++q) {
                    const int4 e = b.ang_slot[q];      // slots of (a, b, c), role in .w
                    const int sa = (int)checked_slot(b.ctl, e.x, b.S, i, kSiteBondSlot),
                              sb = (int)checked_slot(b.ctl, e.y, b.S, i, kSiteBondSlot),
                              sc = (int)checked_slot(b.ctl, e.z, b.S, i, kSiteBondSlot);
                    if (PREC == 1) {
                        const uint4 pa = P[sa], pb = P[sb], pcc = P[sc];
                        const float b1[3] = {(float)(int)(pb.x - pa.x) * R.qs[0], (float)(int)(pb.y - pa.y) * R.qs[1],
                                             (float)(int)(pb.z - pa.z) * R.qs[2]};
                        const float b2[3] = {(float)(int)(pcc.x - pb.x) * R.qs[0], (float)(int)(pcc.y - pb.y) * R.qs[1],
                                             (float)(int)(pcc.z - pb.z) * R.qs[2]};
                        float fa[3], fc[3], u;
                        angle_term<float>(b1, b2, b.angle_K_f, fa, fc, u);
                        // the three visits round F_a and F_c identically and the
                        // middle bead takes minus their sum: the triple adds exactly 0
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const long long qa = fx_round(fa[k]), qc = fx_round(fc[k]);
                            Fd[k] += ll_to_double(e.w == 0 ? qa : (e.w == 2 ? qc : -(qa + qc)));
                        }
                        if (ENERGY) uf += fix_round(2.0 * (double)u / 3.0, 4194304.0);
                    } else {
                        double b1[3], b2[3];
                        for (int k = 0; k < 3; ++k) {
                            double t1 = X[k * b.S + sb] - X[k * b.S + sa];
                            double t2 = X[k * b.S + sc] - X[k * b.S + sb];
                            b1[k] = t1 - R.L[k] * rint(t1 / R.L[k]);
                            b2[k] = t2 - R.L[k] * rint(t2 / R.L[k]);
                        }
                        double fa[3], fc[3], u;
                        angle_term<double>(b1, b2, b.angle_K, fa, fc, u);
                        for (int k = 0; k < 3; ++k) Fd[k] += e.w == 0 ? fa[k] : (e.w == 2 ? fc[k] : -(fa[k] + fc[k]));
                        if (ENERGY) ui += u / 3.0;
                    }
                }
            }
            double v[3];
            if (MODE != kModeOut) {
#pragma unroll
                for (int k = 0; k < 3; ++k) v[k] = b.v[cur][k * b.S + i];
                if (b.langevin) {
                    for (int k = 0; k < 3; ++k) Fd[k] *= fscale;
                    fscale = 1.0;
                    ckick = b.half_dt_over_m;
                    langevin(b, (int)pi.w, step, v, Fd);
                }
            }
            if (MODE == kModeOut) {
                const int id = (int)pi.w;
                if (b.fout)
                    for (int k = 0; k < 3; ++k) b.fout[k * b.N + id] = Fd[k] * fscale;
                if (ENERGY) {
                    double w2 = 0.0;
                    for (int k = 0; k < 3; ++k) { double w = b.v[cur][k * b.S + i]; w2 += w * w; }
                    if (PREC == 1) kf += fix_round(w2, b.mass * 4194304.0);
                    else ki += 0.5 * b.mass * w2;
                }
            } else if (MODE == kModeStore) {
                for (int k = 0; k < 3; ++k) b.F[k * b.S + i] = Fd[k] * fscale;
                if (ENERGY) {
                    const double w2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
                    if (PREC == 1) kf += fix_round(w2, b.mass * 4194304.0);
                    else ki += 0.5 * b.mass * w2;
                }
            } else if (MODE == kModeFinal) {
                const double c = ckick;
                for (int k = 0; k < 3; ++k) {
                    v[k] += c * Fd[k];
                    b.v[cur][k * b.S + i] = v[k];
                    b.F[k * b.S + i] = Fd[k] * fscale;
                }
                if (ENERGY) {
                    const double w2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
                    if (PREC == 1) kf += fix_round(w2, b.mass * 4194304.0);
                    else ki += 0.5 * b.mass * w2;
                }
            } else {  // kModeFused: end of step n, then the first half kick and drift of step n + 1
                const double c = ckick;
                double xi[3];
                for (int k = 0; k < 3; ++k) v[k] += c * Fd[k];
                if (ENERGY) {
                    const double w2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
                    if (PREC == 1) kf += fix_round(w2, b.mass * 4194304.0);
                    else ki += 0.5 * b.mass * w2;
                }
                for (int k = 0; k < 3; ++k) {
                    v[k] += c * Fd[k];
                    xi[k] = X[k * b.S + i];
                }
                ratio = fmaxf(ratio, drift(b, R, i, nxt, pi.w, xi, v));
            }
        };
        // With one particle per thread, the next tile's bulk copies go out as
        // soon as every thread is past its pair sums and arrive during phase 2:
        // each thread arrives on s_p1bar after phase 1 (the copying warp once its
        // copies of the next tile's record are complete); only the first warp
        // waits for all of them, then issues.
        int issued_next = 0;   // the first warp (thread 0 publishes it)
        if (kBulk && Pt <= (int)blockDim.x) {
            PState ps;
            const long long i = tl.s0 + threadIdx.x;
            const bool act = i < tl.s1;
            if (act) phase1(i, ps);
            cp_async_wait_all();   // the next tile's record (the copying warp)
            mbar_arrive(&s_p1bar);
            if (threadIdx.x < 32) {
                if (!mbar_wait(&s_p1bar, p1phase)) err |= kErrTimeout;
                else if (pref) {
                    const int npn = s_npb[buf ^ 1];
                    if (pcb[buf ^ 1][npn].hoff <= b.hcap) {
                        issue_tile_bulk(b, tlb[buf ^ 1], pcb[buf ^ 1], npn, P, hpos, lst, &s_mbar, threadIdx.x);
                        issued_next = 1;
                    }
                }
            }
            p1phase ^= 1u;
            if (act) phase2(i, ps);
        } else {
            for (long long i = tl.s0 + threadIdx.x; i < tl.s1; i += blockDim.x) {
                PState ps;
                phase1(i, ps);
                phase2(i, ps);
            }
        }
        if (ENERGY && PREC != 1) {
            double a = ui, c = ki, d = wi;
            block_sum3(a, c, d, sm3);
            if (threadIdx.x == 0) {
                b.partial[4 * t + 0] = a;
                b.partial[4 * t + 1] = c;
                b.partial[4 * t + 2] = d;
            }
        }
        cp_async_wait_all();   // the next tile's record (the copying warp)
        if (threadIdx.x == 0) {
            s_tile = t_next;
            s_issued = issued_next;
        }
        __syncthreads();   // the halo and the tile record are reused by the next tile
        buf ^= 1;
        have = pref;
    }
    if (ENERGY && PREC == 1 && rcur >= 0) flush_energy(b, rcur, uf, kf, wf, sml);
    if (err) atomicOr(&b.ctl->err, err);
    constexpr bool kDrift = (MODE == kModeFused);
    if (kDrift) ratio = block_max(ratio, smr);
    finish(b, kDrift, ENERGY, true, ratio, PREC == 1);
}

// Pair pass of the half list: the tile loop of k_force (halo and list block
// staged in shared memory), each pair once; a particle's own sum and the
// reactions on its partners go to the fixed-point sums Fq by 64-bit atomic
// adds.  Pair energies and virials per tile (twice the energy, as in the
// full list, where every pair is visited from both ends).  The force kernel
// in its half-list form then reads Fq, integrates and clears it.
template <bool ENERGY>
__global__ void __launch_bounds__(kBlock, MDK_FORCE_MIN_BLOCKS) k_pairs_half(Bufs b)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Piece pc[kMaxPieces + 1];
    __shared__ Tile tl;
    __shared__ int s_tile, s_np, s_self;
    __shared__ int s_nn[kTileMax];
    __shared__ long long sml[kBlock / 32][3];
    if (block_uniform(b.ctl->err != 0)) return;
    const int cur = b.ctl->cur;
    const double *X = b.x[cur];
    const uint4 *P = b.pos[cur];
    uint4 *hpos = reinterpret_cast<uint4 *>(smem_raw);
    unsigned short *lst = reinterpret_cast<unsigned short *>(smem_raw + (size_t)b.hcap * sizeof(uint4));
    int err = 0;
    long long uf = 0, kf = 0, wf = 0;   // summed over this block's tiles until the replica changes
    int rcur = -1;
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(&b.ctl->tile_next, 1u);
    __syncthreads();
    for (;;) {
        const int t = s_tile;
        __syncthreads();
        if (t >= b.ctl->ntiles) break;
        int t_next = 0;
        if (threadIdx.x == 0) t_next = (int)atomicAdd(&b.ctl->tile_next, 1u);
        load_tile(b, t, tl, pc, s_np);
        __syncthreads();
        const Replica &R = b.rep[tl.rep];
        const int np = s_np;
        const int Pt = tl.s1 - tl.s0;
        if (ENERGY && tl.rep != rcur) {   // block-uniform
            if (rcur >= 0) flush_energy(b, rcur, uf, kf, wf, sml);
            rcur = tl.rep;
        }
        if (pc[np].hoff > b.hcap) {
            err |= kErrList;
            if (threadIdx.x == 0) s_tile = t_next;
            __syncthreads();
            continue;
        }
        const bool own_staged = Pt <= kTileMax;
        if (own_staged)
            for (int p = threadIdx.x; p < Pt; p += blockDim.x) cp_async4(&s_nn[p], &b.nn[tl.s0 + p]);
        if (threadIdx.x == 0) s_self = tile_self_offset(R, tl, pc, np);
        stage_halo<uint4>(pc, np, [&](int h, int j) { cp_async16(&hpos[h], &P[j]); });
        const bool lstaged = tl.kmax * Pt <= kListStage * kTileMax;
        if (lstaged) {
            const unsigned short *src = b.nbr + nbr_index(tl.s0, Pt, b.K, 0, 0);
            const int total = tl.kmax * Pt;
            const int nvec = total >> 3;
            const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
            uint4 *d4 = reinterpret_cast<uint4 *>(lst);
            for (int m = threadIdx.x; m < nvec; m += blockDim.x) cp_async16(d4 + m, s4 + m);
            for (int m = (nvec << 3) + threadIdx.x; m < total; m += blockDim.x) lst[m] = src[m];
        }
        cp_async_wait_all();
        __syncthreads();
        // the fourth word of every staged position becomes its slot
        stage_halo<uint4>(pc, np, [&](int h, int j) { hpos[h].w = (unsigned)j; });
        __syncthreads();
        for (long long i = tl.s0 + threadIdx.x; i < tl.s1; i += blockDim.x) {
            const uint4 pi = hpos[checked_entry(b.ctl, s_self + (int)(i - tl.s0), pc[np].hoff, kSiteForceOwn)];
            const int n = min(own_staged ? s_nn[i - tl.s0] : b.nn[i], b.K);
            const int npad = min(((n + kPad - 1) / kPad) * kPad, b.K);
            // a list block too long for the stage is read from global memory
            // through the same [row][particle] layout
            const unsigned short *nbs = lstaged ? lst + (i - tl.s0) : b.nbr + nbr_index(tl.s0, Pt, b.K, 0, (int)(i - tl.s0));
            Acc32 a = {0u, 0u, 0u, 0u, 0u, 0u, make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f), 0};
            if (R.cubic) neighbours32_half<ENERGY, true>(R, hpos, nbs, Pt, n, npad, pi, X, b.S, i, pc, np, a, err, b.Fq, b.ctl,
                                                  pc[np].hoff);
            else neighbours32_half<ENERGY, false>(R, hpos, nbs, Pt, n, npad, pi, X, b.S, i, pc, np, a, err, b.Fq, b.ctl,
                                                   pc[np].hoff);
            const unsigned hs[3] = {a.hx, a.hy, a.hz}, ls[3] = {a.lx, a.ly, a.lz};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const long long v = (long long)(int)hs[k] * 4194304LL + (long long)(int)ls[k];
                if (v != 0) atomicAdd(reinterpret_cast<unsigned long long *>(b.Fq + k * b.S + i), (unsigned long long)v);
            }
            if (ENERGY) {
                // each pair once here: twice its energy and virial, as the
                // full list's two visits give
                uf += fx_round(2.0f * pair_energy(R, a));
                wf += fx_round(2.0f * (R.eps24_f * (a.sg.x + a.sg.y)));
            }
        }
        if (threadIdx.x == 0) s_tile = t_next;
        __syncthreads();   // the halo and the tile record are reused by the next tile
    }
    if (ENERGY && rcur >= 0) flush_energy(b, rcur, uf, kf, wf, sml);
    if (err) atomicOr(&b.ctl->err, err);
    finish(b, false, false, true, 0.0f, true);
}

// Integrate1 of the first step of an md_step call: v += dt/2m F; x += dt v.
__global__ void __launch_bounds__(kBlock) k_kick_drift(Bufs b)
{
    __shared__ float smr[kBlock / 32];
    if (block_uniform(b.ctl->err != 0)) return;
    const int cur = b.ctl->cur, nxt = cur ^ 1;
    const long long i = (long long)blockIdx.x * kBlock + threadIdx.x;
    const Replica &R = b.rep[b.blk_rep[blockIdx.x]];
    float ratio = 0.0f;
    if (i < b.S) {
        uint4 pi = b.pos[cur][i];
        if ((int)pi.w >= 0) {
            double v[3], xi[3];
            for (int k = 0; k < 3; ++k) {
                v[k] = b.v[cur][k * b.S + i] + b.half_dt_over_m * b.F[k * b.S + i];
                xi[k] = b.x[cur][k * b.S + i];
            }
            ratio = drift(b, R, i, nxt, pi.w, xi, v);
        }
    }
    ratio = block_max(ratio, smr);
    finish(b, true, false, false, ratio);
}

// grid of a persistent kernel: resident blocks per SM x SMs
static int persistent_grid(const void *fn, int block, size_t smem)
{
    int dev = 0, nsm = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // the default 48 KB limit covers static plus dynamic shared memory: always opt in
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, block, smem);
    return (occ > 0 ? occ : 1) * (nsm > 0 ? nsm : 1);
}

template <int PREC, int MODE, bool ENERGY, bool HALF>
static void launch_one(const Bufs &b, cudaStream_t st)
{
    // (16 bytes of slack: the bulk copy of a list block rounds up to 16 bytes)
    const size_t smem = HALF ? 0
                             : (size_t)b.hcap * (PREC == 1 ? sizeof(uint4) : 3 * sizeof(double)) +
                                   (size_t)kListStage * kTileMax * sizeof(unsigned short) + 16;
    static int grid = 0;
    static size_t grid_smem = 0;
    if (grid == 0 || grid_smem != smem) {
        grid = persistent_grid((const void *)k_force<PREC, MODE, ENERGY, HALF>, kBlock, smem);
        grid_smem = smem;
    }
    k_force<PREC, MODE, ENERGY, HALF><<<grid, kBlock, smem, st>>>(b);
}

template <bool ENERGY>
static void launch_pairs_half(const Bufs &b, cudaStream_t st)
{
    const size_t smem = (size_t)b.hcap * sizeof(uint4) + (size_t)kListStage * kTileMax * sizeof(unsigned short);
    static int grid = 0;
    static size_t grid_smem = 0;
    if (grid == 0 || grid_smem != smem) {
        grid = persistent_grid((const void *)k_pairs_half<ENERGY>, kBlock, smem);
        grid_smem = smem;
    }
    k_pairs_half<ENERGY><<<grid, kBlock, smem, st>>>(b);
}

template <int PREC, bool HALF>
static void launch_force_p(const Bufs &b, int mode, bool energy, cudaStream_t st)
{
#define MDK_CASE(M)                                              \
    case M:                                                      \
        if (energy) launch_one<PREC, M, true, HALF>(b, st);      \
        else launch_one<PREC, M, false, HALF>(b, st);            \
        break;
    switch (mode) {
        MDK_CASE(kModeOut)
        MDK_CASE(kModeStore)
        MDK_CASE(kModeFused)
        MDK_CASE(kModeFinal)
        default: break;
    }
#undef MDK_CASE
}

// One force evaluation in the given mode.  With a half list (FP32 only) it
// is two kernels: the pair pass into the fixed-point sums, then the force
// kernel's half-list form, which integrates from them.
void launch_force(const Bufs &b, int precision, int mode, bool energy, cudaStream_t st)
{
    if (precision == 1 && b.half_list) {
        if (energy) launch_pairs_half<true>(b, st);
        else launch_pairs_half<false>(b, st);
        launch_force_p<1, true>(b, mode, energy, st);
    } else if (precision == 1) launch_force_p<1, false>(b, mode, energy, st);
    else launch_force_p<0, false>(b, mode, energy, st);
}

void launch_kick_drift(const Bufs &b, cudaStream_t st) { k_kick_drift<<<b.nblk, kBlock, 0, st>>>(b); }

// The bounded wait of the tile kernels on a barrier that no arrival and no
// copy will complete: every thread gives up after `polls` polls and the
// block latches the timeout, as a block whose bulk copies never arrived does.
__global__ void __launch_bounds__(kBlock) k_wait_selftest(Bufs b, int polls)
{
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    const bool late = !mbar_wait(&bar, 0u, polls);
    if (__syncthreads_or(late) && threadIdx.x == 0) atomicOr(&b.ctl->err, kErrTimeout);
}

void launch_wait_selftest(const Bufs &b, int polls, cudaStream_t st) { k_wait_selftest<<<1, kBlock, 0, st>>>(b, polls); }

}  // namespace mdk
