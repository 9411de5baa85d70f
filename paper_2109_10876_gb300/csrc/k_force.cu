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
#include "md_internal.cuh"

namespace mdk {

constexpr float kMagic = 12582912.0f;       // 1.5 * 2^23: x + kMagic rounds x to an integer
constexpr unsigned kMagicBits = 0x4B400000u;
constexpr float kFixScale = 4194304.0f;     // 2^22
constexpr double kFixInv = 1.0 / 4194304.0;
#ifndef MDK_GATHER_BATCH
#define MDK_GATHER_BATCH 4
#endif
#ifndef MDK_FORCE_MIN_BLOCKS
#define MDK_FORCE_MIN_BLOCKS 6
#endif
constexpr int kU = MDK_GATHER_BATCH;         // neighbours gathered per batch

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

__device__ __forceinline__ double fx_value(unsigned hi, unsigned lo)
{
    long long v = (long long)(int)hi * 4194304LL + (long long)(int)lo;
    return (double)v * kFixInv;
}

__device__ __forceinline__ unsigned to_q2(double y, double scale)
{
    long long q = __double2ll_rn(y * scale);
    return (unsigned)(q & 0xffffffffLL);
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

// Last block: per-replica totals from the block partials, in a fixed order.
__device__ void reduce_partials(const Bufs &b, double *thermo)
{
    __shared__ double red[kBlock][3];
    for (int r = 0; r < b.nrep; ++r) {
        const Replica &R = b.rep[r];
        double a = 0, c = 0, d = 0;
        for (int q = R.blk_begin + threadIdx.x; q < R.blk_end; q += blockDim.x) {
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
        long long qq = __double2ll_rn(y * R.to_q[k]);
        if ((unsigned long long)qq >= 4294967296ULL) {
            y = wrap1(y, R.L[k]);
            qq = __double2ll_rn(y * R.to_q[k]);
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

// End-of-kernel bookkeeping by the last block to finish: energy totals, and
// for kernels that drifted, the buffer flip, the step counter and the
// rebuild decision for the next step.
__device__ void finish(const Bufs &b, bool drifted, bool energy, float ratio_blk)
{
    if (!drifted && !energy) return;
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
    if (energy) reduce_partials(b, b.thermo);
    if (threadIdx.x == 0) {
        if (drifted) {
            unsigned bits = atomicExch(&b.ctl->disp2_bits, 0u);
            b.ctl->rebuild = (__uint_as_float(bits) > 1.0f) ? 1 : 0;
            b.ctl->cur ^= 1;
            b.ctl->step += 1;
        }
        b.ctl->done_force = 0u;
    }
}

// FP32 pair terms of one neighbour: separation from the fixed-point
// positions, LJ force scalar masked to zero outside the cutoff, and the
// fixed-point accumulation.  `in` decides membership; the caller passes the
// FP32 verdict or, for the rare pairs within rounding of r_cut, the FP64 one.
struct Acc32 {
    unsigned hx, lx, hy, ly, hz, lz, hu, lu, hw, lw;
};

template <bool ENERGY>
__device__ __forceinline__ void pair32(float dx, float dy, float dz, float r2, bool in, float sig2, float eps24,
                                       float eps4, float vsh, Acc32 &a)
{
    const float ir2 = rcp_approx(r2);
    const float s2 = sig2 * ir2;
    const float s6 = s2 * s2 * s2;
    const float fs = in ? eps24 * s6 * (2.0f * s6 - 1.0f) * ir2 : 0.0f;
    fx_acc2(fs, dx, a.hx, a.lx);
    fx_acc2(fs, dy, a.hy, a.ly);
    fx_acc2(fs, dz, a.hz, a.lz);
    if (ENERGY) {
        fx_acc(in ? eps4 * s6 * (s6 - 1.0f) - vsh : 0.0f, a.hu, a.lu);
        fx_acc2(fs, r2, a.hw, a.lw);
    }
}

template <int PREC, int MODE, bool ENERGY>
__global__ void __launch_bounds__(kBlock, PREC == 1 ? MDK_FORCE_MIN_BLOCKS : 1) k_force(Bufs b)
{
    __shared__ double sm3[kBlock / 32][3];
    __shared__ float smr[kBlock / 32];
    if (b.ctl->err) return;
    const int cur = b.ctl->cur, nxt = cur ^ 1;
    const long long step = b.ctl->step;
    const long long i = (long long)blockIdx.x * kBlock + threadIdx.x;
    const Replica &R = b.rep[b.blk_rep[blockIdx.x]];
    const double *X = b.x[cur];
    // Fd * fscale is the force; FP32 mode keeps the exact fixed-point integer
    // in Fd so that the 2^-22 scale folds into the kick constant
    double Fd[3] = {0.0, 0.0, 0.0};
    double fscale = 1.0;
    double ui = 0.0, wi = 0.0, ki = 0.0;
    float ratio = 0.0f;
    uint4 pi = make_uint4(0u, 0u, 0u, 0xffffffffu);
    bool real = false;
    int err = 0;
    if (i < b.S) {
        pi = b.pos[cur][i];
        real = (int)pi.w >= 0;
    }
    if (real) {
        const int n = min(b.nn[i], b.K);
        const int *nb = b.nbr + nbr_index(i, 0, b.K);   // entry k at nb[32 k]
        if (PREC == 1) {
            const uint4 *P = b.pos[cur];
            const float qs0 = R.qs[0], qs1 = R.qs[1], qs2 = R.qs[2];
            const float rc2_lo = R.rc2_lo, rc2_hi = R.rc2_hi, fmax2 = R.fmax2;
            const float sig2 = R.sig2_f, eps24 = R.eps24_f, eps4 = R.eps4_f, vsh = R.vshift_f;
            // a point half a box away on every axis: never within the cutoff
            const uint4 far = make_uint4(pi.x ^ 0x80000000u, pi.y ^ 0x80000000u, pi.z ^ 0x80000000u, 0u);
            Acc32 a = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
            int nband = 0;
            bool tooclose = false;
            // neighbours in batches of kU: all index loads, then all position
            // gathers, then branch-free arithmetic
            for (int k0 = 0; k0 < n; k0 += kU) {
                int jj[kU];
                uint4 pj[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) jj[u] = (k0 + u < n) ? __ldg(nb + 32 * (k0 + u)) : 0;
#pragma unroll
                for (int u = 0; u < kU; ++u) pj[u] = (k0 + u < n) ? __ldg(P + jj[u]) : far;
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const float dx = (float)(int)(pi.x - pj[u].x) * qs0;
                    const float dy = (float)(int)(pi.y - pj[u].y) * qs1;
                    const float dz = (float)(int)(pi.z - pj[u].z) * qs2;
                    const float r2 = dx * dx + dy * dy + dz * dz;
                    const bool in = r2 < rc2_lo;
                    nband += (r2 < rc2_hi) & !in;
                    tooclose |= r2 < fmax2;
                    pair32<ENERGY>(dx, dy, dz, r2, in, sig2, eps24, eps4, vsh, a);
                }
            }
            if (nband) {
                // pairs within rounding of r_cut: membership decided in FP64
                // from the master positions, as in the FP64 reference
                for (int k = 0; k < n; ++k) {
                    const int j = __ldg(nb + 32 * k);
                    const uint4 q = __ldg(P + j);
                    const float dx = (float)(int)(pi.x - q.x) * qs0;
                    const float dy = (float)(int)(pi.y - q.y) * qs1;
                    const float dz = (float)(int)(pi.z - q.z) * qs2;
                    const float r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 >= rc2_lo && r2 < rc2_hi && r2_exact(X, b.S, i, j, R.L) < R.rc2)
                        pair32<ENERGY>(dx, dy, dz, r2, true, sig2, eps24, eps4, vsh, a);
                }
            }
            if (tooclose) err |= kErrFixed;
            const unsigned hh[3] = {a.hx, a.hy, a.hz}, ll[3] = {a.lx, a.ly, a.lz};
#pragma unroll
            for (int k = 0; k < 3; ++k)
                Fd[k] = (double)((long long)(int)hh[k] * 4194304LL + (long long)(int)ll[k]);
            fscale = kFixInv;
            if (ENERGY) { ui = 0.5 * fx_value(a.hu, a.lu); wi = 0.5 * fx_value(a.hw, a.lw); }
        } else {
            const double xi0 = X[i], xi1 = X[b.S + i], xi2 = X[2 * b.S + i];
            const double L0 = R.L[0], L1 = R.L[1], L2 = R.L[2];
            const double h0 = 0.5 * L0, h1 = 0.5 * L1, h2 = 0.5 * L2;
            const double eps24 = 24.0 * R.eps, eps4 = 4.0 * R.eps, sig2 = R.sigma * R.sigma;
            const double rc2 = R.rc2, vsh = R.vshift;
            const double band = 1e-12 * rc2;
            for (int k0 = 0; k0 < n; k0 += kU) {
                int jj[kU];
                double xj[kU][3];
#pragma unroll
                for (int u = 0; u < kU; ++u) jj[u] = (k0 + u < n) ? __ldg(nb + 32 * (k0 + u)) : -1;
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const long long j = jj[u] >= 0 ? jj[u] : i;
                    xj[u][0] = __ldg(X + j);
                    xj[u][1] = __ldg(X + b.S + j);
                    xj[u][2] = __ldg(X + 2 * b.S + j);
                }
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    double dx = xi0 - xj[u][0], dy = xi1 - xj[u][1], dz = xi2 - xj[u][2];
                    dx = dx > h0 ? dx - L0 : (dx < -h0 ? dx + L0 : dx);
                    dy = dy > h1 ? dy - L1 : (dy < -h1 ? dy + L1 : dy);
                    dz = dz > h2 ? dz - L2 : (dz < -h2 ? dz + L2 : dz);
                    const double r2 = dx * dx + dy * dy + dz * dz;
                    if (jj[u] >= 0 && r2 < rc2 + band) {
                        bool in = r2 < rc2 - band;
                        if (!in) in = r2_exact(X, b.S, i, jj[u], R.L) < rc2;
                        if (in) {
                            const double ir2 = 1.0 / r2;
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
            }
            if (!isfinite(Fd[0]) || !isfinite(Fd[1]) || !isfinite(Fd[2])) err |= kErrNonfinite;
        }
        // FENE bonds of this particle (Sec. 4), both ends of every bond visited;
        // in FP32 mode the bond force joins the same fixed-point sum
        if (b.has_bonds) {
            const int id = (int)pi.w;
            for (int q = b.bond_off[id]; q < b.bond_off[id + 1]; ++q) {
                const int sj = b.slot_of_id[b.bond_partner[q]];
                if (PREC == 1) {
                    const uint4 pj = b.pos[cur][sj];
                    const float dx = (float)(int)(pi.x - pj.x) * R.qs[0];
                    const float dy = (float)(int)(pi.y - pj.y) * R.qs[1];
                    const float dz = (float)(int)(pi.z - pj.z) * R.qs[2];
                    const float r2 = dx * dx + dy * dy + dz * dz;
                    const float qf = 1.0f - r2 / b.fene_R02_f;
                    if (!(qf > 0.0f)) { err |= kErrBond; continue; }
                    const float c = -b.fene_K_f / qf;
                    unsigned h = 0, l = 0;
                    fx_acc2(c, dx, h, l); Fd[0] += (double)((long long)(int)h * 4194304LL + (long long)(int)l); h = l = 0;
                    fx_acc2(c, dy, h, l); Fd[1] += (double)((long long)(int)h * 4194304LL + (long long)(int)l); h = l = 0;
                    fx_acc2(c, dz, h, l); Fd[2] += (double)((long long)(int)h * 4194304LL + (long long)(int)l);
                    if (ENERGY) {
                        ui += 0.5 * (-0.5 * b.fene_K * b.fene_R02 * log((double)qf));
                        wi += 0.5 * (double)(c * r2);
                    }
                } else {
                    double d[3];
                    for (int k = 0; k < 3; ++k) {
                        double t = X[k * b.S + i] - X[k * b.S + sj];
                        d[k] = t - R.L[k] * rint(t / R.L[k]);
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

        double v[3];
        if (MODE != kModeOut) {
#pragma unroll
            for (int k = 0; k < 3; ++k) v[k] = b.v[cur][k * b.S + i];
            if (b.langevin) {
                for (int k = 0; k < 3; ++k) Fd[k] *= fscale;
                fscale = 1.0;
                langevin(b, (int)pi.w, step, v, Fd);
            }
        }
        if (MODE == kModeOut) {
            const int id = (int)pi.w;
            if (b.fout)
                for (int k = 0; k < 3; ++k) b.fout[k * b.N + id] = Fd[k] * fscale;
            if (ENERGY)
                for (int k = 0; k < 3; ++k) { double w = b.v[cur][k * b.S + i]; ki += 0.5 * b.mass * w * w; }
        } else if (MODE == kModeStore) {
            for (int k = 0; k < 3; ++k) b.F[k * b.S + i] = Fd[k] * fscale;
            if (ENERGY) for (int k = 0; k < 3; ++k) ki += 0.5 * b.mass * v[k] * v[k];
        } else if (MODE == kModeFinal) {
            const double c = b.half_dt_over_m * fscale;
            for (int k = 0; k < 3; ++k) {
                v[k] += c * Fd[k];
                b.v[cur][k * b.S + i] = v[k];
                b.F[k * b.S + i] = Fd[k] * fscale;
                if (ENERGY) ki += 0.5 * b.mass * v[k] * v[k];
            }
        } else {  // kModeFused: end of step n and first half kick of step n + 1
            const double c = b.half_dt_over_m * fscale;
            double xi[3];
            for (int k = 0; k < 3; ++k) {
                v[k] += c * Fd[k];                        // synchronised v_n
                if (ENERGY) ki += 0.5 * b.mass * v[k] * v[k];
                v[k] += c * Fd[k];
                xi[k] = X[k * b.S + i];
            }
            ratio = drift(b, R, i, nxt, pi.w, xi, v);
        }
    } else if (MODE == kModeFused && i < b.S) {
        b.pos[nxt][i] = pi;   // padding slot: keep the id marker in the other buffer
    }
    if (err) atomicOr(&b.ctl->err, err);

    if (ENERGY) {
        double a = ui, c = ki, d = wi;
        block_sum3(a, c, d, sm3);
        if (threadIdx.x == 0) {
            b.partial[4 * blockIdx.x + 0] = a;
            b.partial[4 * blockIdx.x + 1] = c;
            b.partial[4 * blockIdx.x + 2] = d;
        }
    }
    constexpr bool kDrift = (MODE == kModeFused);
    if (kDrift) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ratio = fmaxf(ratio, __shfl_xor_sync(0xffffffffu, ratio, o));
        if ((threadIdx.x & 31) == 0) smr[threadIdx.x >> 5] = ratio;
        __syncthreads();
        if (threadIdx.x == 0)
            for (int q = 1; q < kBlock / 32; ++q) ratio = fmaxf(ratio, smr[q]);
    }
    finish(b, kDrift, ENERGY, ratio);
}

// Integrate1 of the first step of an md_step call: v += dt/2m F; x += dt v.
__global__ void __launch_bounds__(kBlock) k_kick_drift(Bufs b)
{
    __shared__ float smr[kBlock / 32];
    if (b.ctl->err) return;
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
        } else {
            b.pos[nxt][i] = pi;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ratio = fmaxf(ratio, __shfl_xor_sync(0xffffffffu, ratio, o));
    if ((threadIdx.x & 31) == 0) smr[threadIdx.x >> 5] = ratio;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int q = 1; q < kBlock / 32; ++q) ratio = fmaxf(ratio, smr[q]);
    finish(b, true, false, ratio);
}

template <int PREC>
static void launch_force_p(const Bufs &b, int mode, bool energy, cudaStream_t st)
{
#define MDK_CASE(M)                                                                         \
    case M:                                                                                 \
        if (energy) k_force<PREC, M, true><<<b.nblk, kBlock, 0, st>>>(b);                   \
        else k_force<PREC, M, false><<<b.nblk, kBlock, 0, st>>>(b);                         \
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

void launch_force(const Bufs &b, int precision, int mode, bool energy, cudaStream_t st)
{
    if (precision == 1) launch_force_p<1>(b, mode, energy, st);
    else launch_force_p<0>(b, mode, energy, st);
}

void launch_kick_drift(const Bufs &b, cudaStream_t st) { k_kick_drift<<<b.nblk, kBlock, 0, st>>>(b); }

}  // namespace mdk
