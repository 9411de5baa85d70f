// Adjoint kernels for reverse-mode differentiation through velocity Verlet
// (NVE, pair potential of Eq. 2; arXiv:2109.10876 Fig. 1 gives the map being
// differentiated).  For a loss L(U, K, W) of the final state the reverse pass
// needs, at recorded positions x:
//   the Hessian-vector product of the pair forces, (J w)_i = sum_j
//     [g (w_i - w_j) + (g'/r) d (d . (w_i - w_j))],  f_ij = g(r) d,
//   the parameter projections sum_i w_i . dF_i/deps = sum_i w_i . F_i / eps and
//     sum_i w_i . dF_i/dsigma = sum_i w_i . sum_j (dg/dsigma) d,
// and, at the final state, F, dW/dx, U, W and sum_pairs r^2 dg/dsigma.
// All in FP64, over the Verlet lists of the forward machinery (tiles, halo in
// shared memory).  Vectors w, J w and the adjoints live in the caller's
// particle order; kernels map through the particle id in pos.w.
#include <algorithm>

#include "md_internal.cuh"

namespace mdk {

__device__ __noinline__ double adj_r2_exact(const double *x, long long S, long long i, long long j, const double *L)
{
    double d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double t = __dsub_rn(x[k * S + i], x[k * S + j]);
        const double q = rint(__ddiv_rn(t, L[k]));
        d[k] = __dsub_rn(t, __dmul_rn(L[k], q));
    }
    return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

__device__ __forceinline__ int adj_halo_slot(const Piece *pc, int np, int h)
{
    int q = 0;
    while (q + 1 < np && h >= pc[q + 1].hoff) ++q;
    return pc[q].slot0 + (h - pc[q].hoff);
}

// bounds check of the checked build (md_ok): v within [0, lim), else 0
__device__ __forceinline__ long long adj_checked(Ctl *ctl, long long v, long long lim)
{
    return md_ok(ctl, v >= 0 && v < lim, kSiteAdjHalo, v) ? v : 0;
}

// Last block: per-replica sums of the 4 per-tile partials, added into
// acc[4 * r + k] with weight `scale`.  Each warp takes every fourth replica:
// lane-strided sums over its tiles, then a shuffle tree (a fixed order, so
// the result does not depend on timing); no block barriers.
__device__ void adj_reduce(const Bufs &b, double scale, double *acc)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int r = warp; r < b.nrep; r += nwarp) {
        double a[4] = {0, 0, 0, 0};
        for (int q = b.rep_tile[r] + lane; q < b.rep_tile[r + 1]; q += 32)
            for (int k = 0; k < 4; ++k) a[k] += b.partial[4 * q + k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            for (int k = 0; k < 4; ++k) a[k] += __shfl_down_sync(0xffffffffu, a[k], o);
        if (lane == 0)
            for (int k = 0; k < 4; ++k) acc[4 * r + k] += scale * a[k];
    }
}

// MODE 0 (HVP): hv = J w at the current positions; partials (w.F/eps, w.dF/dsigma).
// MODE 1 (LOSS): lx = -cU F + cW dW/dx, lv = cK m v; partials (U, W, sum r^2 dg/dsigma).
// coef: per replica (cU, cK, cW, -) for LOSS; the partials are added into
// acc (4 per replica) with weight `scale`.
template <int MODE>
__global__ void __launch_bounds__(kBlock) k_adj(Bufs b, const double *w, double *out0, double *out1,
                                                const double *coef, double scale, double *acc)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Piece pc[kMaxPieces + 1];
    __shared__ Tile tl;
    __shared__ int s_tile, s_np;
    __shared__ double sm4[kBlock / 32][4];
    __shared__ bool last;
    if (block_uniform(b.ctl->err != 0)) return;
    const int cur = b.ctl->cur;
    const double *X = b.x[cur];
    const uint4 *P = b.pos[cur];
    double *hx = reinterpret_cast<double *>(smem_raw);
    double *hy = hx + b.hcap, *hz = hy + b.hcap;
    double *hw = hz + b.hcap;                     // 3 * hcap: w of the halo (MODE 0)
    for (;;) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(&b.ctl->tile_next, 1u);
        __syncthreads();
        const int t = s_tile;
        if (t >= b.ctl->ntiles) break;
        load_tile(b, t, tl, pc, s_np);
        __syncthreads();
        const Replica &R = b.rep[tl.rep];
        const int np = s_np;
        const int Pt = tl.s1 - tl.s0;
        stage_halo<double>(pc, np, [&](int h, int j) {
            hx[h] = X[j];
            hy[h] = X[b.S + j];
            hz[h] = X[2 * b.S + j];
            if (MODE == 0) {
                const int id = (int)adj_checked(b.ctl, (int)P[j].w, b.N);
                hw[3 * h + 0] = w[id];
                hw[3 * h + 1] = w[b.N + id];
                hw[3 * h + 2] = w[2 * b.N + id];
            }
        });
        __syncthreads();
        const double L0 = R.L[0], L1 = R.L[1], L2 = R.L[2];
        const double h0 = 0.5 * L0, h1 = 0.5 * L1, h2 = 0.5 * L2;
        const double eps = R.eps, sig = R.sigma, sig2 = sig * sig, rc2 = R.rc2;
        const double eps24 = 24.0 * eps, isig = 1.0 / sig;
        const double band = 1e-12 * rc2;
        double p0 = 0.0, p1 = 0.0, p2 = 0.0;
        for (long long i = tl.s0 + threadIdx.x; i < tl.s1; i += blockDim.x) {
            const int id = (int)adj_checked(b.ctl, (int)P[i].w, b.N);
            const int n = min(b.nn[i], b.K);
            const unsigned short *nb = b.nbr + nbr_index(tl.s0, Pt, b.K, 0, (int)(i - tl.s0));
            const double xi0 = X[i], xi1 = X[b.S + i], xi2 = X[2 * b.S + i];
            double wi[3] = {0, 0, 0};
            if (MODE == 0) { wi[0] = w[id]; wi[1] = w[b.N + id]; wi[2] = w[2 * b.N + id]; }
            double acc3[3] = {0, 0, 0}, F[3] = {0, 0, 0}, Fs[3] = {0, 0, 0};
            double u = 0.0, wv = 0.0, ws = 0.0;
            for (int k = 0; k < n; ++k) {
                const int h = (int)adj_checked(b.ctl, __ldg(nb + (long long)k * Pt), pc[np].hoff);
                double dx = xi0 - hx[h], dy = xi1 - hy[h], dz = xi2 - hz[h];
                dx = dx > h0 ? dx - L0 : (dx < -h0 ? dx + L0 : dx);
                dy = dy > h1 ? dy - L1 : (dy < -h1 ? dy + L1 : dy);
                dz = dz > h2 ? dz - L2 : (dz < -h2 ? dz + L2 : dz);
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (!(r2 < rc2 + band)) continue;
                if (!(r2 < rc2 - band) &&
                    !(adj_r2_exact(X, b.S, i, adj_checked(b.ctl, adj_halo_slot(pc, np, h), b.S), R.L) < rc2))
                    continue;
                // 1/r^2 by the reciprocal approximation and two Newton steps (the
                // IEEE divide is a long sequence on the narrow FP64 pipe)
                const double ir2 = rcp_newton(r2);
                const double s2 = sig2 * ir2, s6 = s2 * s2 * s2, s12 = s6 * s6;
                const double e24 = eps24 * ir2;
                const double g = e24 * (2.0 * s12 - s6);
                const double gpr = e24 * ir2 * (8.0 * s6 - 28.0 * s12);
                const double dgds = e24 * isig * (24.0 * s12 - 6.0 * s6);
                const double d[3] = {dx, dy, dz};
                if (MODE == 0) {
                    const double dw[3] = {wi[0] - hw[3 * h], wi[1] - hw[3 * h + 1], wi[2] - hw[3 * h + 2]};
                    const double ddw = dx * dw[0] + dy * dw[1] + dz * dw[2];
                    for (int q = 0; q < 3; ++q) {
                        acc3[q] += g * dw[q] + gpr * d[q] * ddw;
                        F[q] += g * d[q];
                        Fs[q] += dgds * d[q];
                    }
                } else {
                    for (int q = 0; q < 3; ++q) {
                        F[q] += g * d[q];
                        acc3[q] += (2.0 * g + gpr * r2) * d[q];      // dW/dx_i
                    }
                    u += 0.5 * (4.0 * eps * (s12 - s6) - R.vshift);
                    wv += 0.5 * g * r2;
                    ws += 0.5 * r2 * dgds;
                }
            }
            if (MODE == 0) {
                for (int q = 0; q < 3; ++q) out0[q * b.N + id] = acc3[q];
                p0 += (wi[0] * F[0] + wi[1] * F[1] + wi[2] * F[2]) / eps;
                p1 += wi[0] * Fs[0] + wi[1] * Fs[1] + wi[2] * Fs[2];
            } else {
                const double cU = coef[4 * tl.rep], cK = coef[4 * tl.rep + 1], cW = coef[4 * tl.rep + 2];
                for (int q = 0; q < 3; ++q) {
                    out0[q * b.N + id] = -cU * F[q] + cW * acc3[q];
                    out1[q * b.N + id] = cK * b.mass * b.v[cur][q * b.S + i];
                }
                p0 += u;
                p1 += wv;
                p2 += ws;
            }
        }
        // per-tile partials in a fixed order
        for (int o = 16; o > 0; o >>= 1) {
            p0 += __shfl_down_sync(0xffffffffu, p0, o);
            p1 += __shfl_down_sync(0xffffffffu, p1, o);
            p2 += __shfl_down_sync(0xffffffffu, p2, o);
        }
        if ((threadIdx.x & 31) == 0) { sm4[threadIdx.x >> 5][0] = p0; sm4[threadIdx.x >> 5][1] = p1; sm4[threadIdx.x >> 5][2] = p2; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0, c = 0, d = 0;
            for (int q = 0; q < kBlock / 32; ++q) { a += sm4[q][0]; c += sm4[q][1]; d += sm4[q][2]; }
            b.partial[4 * t + 0] = a;
            b.partial[4 * t + 1] = c;
            b.partial[4 * t + 2] = d;
            b.partial[4 * t + 3] = 0.0;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        last = (atomicAdd(&b.ctl->done_force, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    adj_reduce(b, scale, acc);
    if (threadIdx.x == 0) {
        b.ctl->tile_next = 0u;
        b.ctl->done_force = 0u;
    }
}

// Reciprocal by the hardware approximation (a pure function of its input).
__device__ __forceinline__ float rcp_approx_f(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// w (caller order, FP64) into slot order as FP32 (hi, lo) pieces, so that the
// halo staging of k_adj_hvp32 copies contiguous runs instead of gathering and
// converting w for every halo entry.
__global__ void k_adj_wslots(Bufs b, const double *w)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.S) return;
    const int id = (int)b.pos[b.ctl->cur][s].w;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 c = make_float2(0.f, 0.f);
    if (id >= 0) {
        const double w0 = w[id], w1 = w[b.N + id], w2 = w[2 * b.N + id];
        const float a0 = (float)w0, a1 = (float)w1, a2 = (float)w2;
        a = make_float4(a0, a1, a2, (float)(w0 - (double)a0));
        c = make_float2((float)(w1 - (double)a1), (float)(w2 - (double)a2));
    }
    b.adj_wa[s] = a;
    b.adj_wb[s] = c;
}

// Hessian-vector product for the FP32 + fixed-point forward path (MODE 0 of
// k_adj in FP32): separations from the fixed-point positions as in the force
// kernel, the interacting set decided the same way (FP64 within rounding of
// r_cut), pair terms and per-particle sums in FP32, w staged as FP32 (hi, lo)
// pairs so that w_i - w_j keeps about 48 bits.  The adjoint state itself
// (lx, lv) and the parameter projections stay FP64.
// Staged like the force kernel: the first warp copies the tile's halo
// positions and list block by bulk (TMA) copies onto an mbarrier (a bounded
// wait); the fourth word of each staged position is then replaced by its slot,
// where the entry's w pieces are read.  The pair loop takes two neighbours at
// a time with packed FP32 instructions and no branches: entries beyond r_cut
// (and the padding) are masked, and their w is not read; entries within FP32
// rounding of r_cut are settled afterwards in FP64.

// The pair terms of one neighbour (scalar) or two (packed), added into the
// per-particle sums: acc += g dw + g' (d.dw) d, F += g d, Fs += dg/dsigma d,
// with g = 24 eps (2 s^12 - s^6) / r^2.
struct HvpSums {
    float2 ax, ay, az, fx, fy, fz, sx, sy, sz;
};

// a - b for two lanes (the negation is exact)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

__device__ __forceinline__ void hvp_pair2(float2 dx, float2 dy, float2 dz, float2 ir2, float4 wa0, float2 wb0,
                                          float4 wa1, float2 wb1, const float4 &wai, const float2 &wbi, float sig2,
                                          float eps24, float isig, HvpSums &a)
{
    const float2 s2 = __fmul2_rn(make_float2(sig2, sig2), ir2);
    const float2 s6 = __fmul2_rn(__fmul2_rn(s2, s2), s2);
    const float2 s12 = __fmul2_rn(s6, s6);
    const float2 e24 = __fmul2_rn(make_float2(eps24, eps24), ir2);
    const float2 g = __fmul2_rn(e24, __ffma2_rn(make_float2(2.0f, 2.0f), s12, make_float2(-s6.x, -s6.y)));
    const float2 gpr = __fmul2_rn(__fmul2_rn(e24, ir2),
                                  __ffma2_rn(make_float2(8.0f, 8.0f), s6, __fmul2_rn(make_float2(-28.0f, -28.0f), s12)));
    const float2 dgds = __fmul2_rn(__fmul2_rn(e24, make_float2(isig, isig)),
                                   __ffma2_rn(make_float2(24.0f, 24.0f), s12, __fmul2_rn(make_float2(-6.0f, -6.0f), s6)));
    // w_i - w_j from the (hi, lo) pieces
    const float2 dwx = __fadd2_rn(sub2(make_float2(wai.x, wai.x), make_float2(wa0.x, wa1.x)),
                                  sub2(make_float2(wai.w, wai.w), make_float2(wa0.w, wa1.w)));
    const float2 dwy = __fadd2_rn(sub2(make_float2(wai.y, wai.y), make_float2(wa0.y, wa1.y)),
                                  sub2(make_float2(wbi.x, wbi.x), make_float2(wb0.x, wb1.x)));
    const float2 dwz = __fadd2_rn(sub2(make_float2(wai.z, wai.z), make_float2(wa0.z, wa1.z)),
                                  sub2(make_float2(wbi.y, wbi.y), make_float2(wb0.y, wb1.y)));
    const float2 ddw = __ffma2_rn(dz, dwz, __ffma2_rn(dy, dwy, __fmul2_rn(dx, dwx)));
    const float2 gd = __fmul2_rn(gpr, ddw);
    a.ax = __fadd2_rn(a.ax, __ffma2_rn(g, dwx, __fmul2_rn(gd, dx)));
    a.ay = __fadd2_rn(a.ay, __ffma2_rn(g, dwy, __fmul2_rn(gd, dy)));
    a.az = __fadd2_rn(a.az, __ffma2_rn(g, dwz, __fmul2_rn(gd, dz)));
    a.fx = __ffma2_rn(g, dx, a.fx);
    a.fy = __ffma2_rn(g, dy, a.fy);
    a.fz = __ffma2_rn(g, dz, a.fz);
    a.sx = __ffma2_rn(dgds, dx, a.sx);
    a.sy = __ffma2_rn(dgds, dy, a.sy);
    a.sz = __ffma2_rn(dgds, dz, a.sz);
}

// One particle's HVP sums from its list (entry k at nb[k Pt]: the staged list
// block when LSMEM, else the list in global memory).
template <bool LSMEM>
__device__ __forceinline__ void hvp_particle(const Bufs &b, const Replica &R, const uint4 *hpos, int H,
                                             const unsigned short *nb, int Pt, int n, int npad, uint4 pi,
                                             long long i, const float4 &wai, const float2 &wbi, HvpSums &a)
{
    const float qs0 = R.qs[0], qs1 = R.qs[1], qs2 = R.qs[2];
    const float lo = R.rc2_lo, hi = R.rc2_hi;
    const float eps24 = 24.0f * (float)R.eps, sig2 = (float)(R.sigma * R.sigma), isig = (float)(1.0 / R.sigma);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float2 z2 = make_float2(0.f, 0.f);
    bool band = false;   // a pair within rounding of r_cut
    for (int k0 = 0; k0 < npad; k0 += 4) {
        int hh[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            hh[u] = (int)adj_checked(b.ctl, LSMEM ? nb[(k0 + u) * Pt] : __ldg(nb + (long long)(k0 + u) * Pt), H);
#pragma unroll
        for (int u = 0; u < 4; u += 2) {
            const uint4 q0 = lds128(hpos + hh[u]), q1 = lds128(hpos + hh[u + 1]);
            const float2 dx = __fmul2_rn(make_float2((float)(int)(pi.x - q0.x), (float)(int)(pi.x - q1.x)),
                                         make_float2(qs0, qs0));
            const float2 dy = __fmul2_rn(make_float2((float)(int)(pi.y - q0.y), (float)(int)(pi.y - q1.y)),
                                         make_float2(qs1, qs1));
            const float2 dz = __fmul2_rn(make_float2((float)(int)(pi.z - q0.z), (float)(int)(pi.z - q1.z)),
                                         make_float2(qs2, qs2));
            const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
            // padding entries are the particle itself (r^2 = 0)
            const bool in0 = (r2.x < lo) & (r2.x > 0.0f), in1 = (r2.y < lo) & (r2.y > 0.0f);
            band |= ((r2.x < hi) & !(r2.x < lo)) | ((r2.y < hi) & !(r2.y < lo));
            float2 ir2 = make_float2(rcp_approx_f(r2.x), rcp_approx_f(r2.y));
            ir2.x = in0 ? ir2.x : 0.0f;
            ir2.y = in1 ? ir2.y : 0.0f;
            const long long j0 = adj_checked(b.ctl, (long long)q0.w, b.S), j1 = adj_checked(b.ctl, (long long)q1.w, b.S);
            const float4 wa0 = in0 ? __ldg(b.adj_wa + j0) : z4, wa1 = in1 ? __ldg(b.adj_wa + j1) : z4;
            const float2 wb0 = in0 ? __ldg(b.adj_wb + j0) : z2, wb1 = in1 ? __ldg(b.adj_wb + j1) : z2;
            hvp_pair2(dx, dy, dz, ir2, wa0, wb0, wa1, wb1, wai, wbi, sig2, eps24, isig, a);
        }
    }
    if (band) {
        // pairs within rounding of r_cut: membership decided in FP64 from the
        // master positions; each as one lane of a packed pair (the other masked)
        for (int k = 0; k < n; ++k) {
            const int h = (int)adj_checked(b.ctl, LSMEM ? nb[k * Pt] : __ldg(nb + (long long)k * Pt), H);
            const uint4 q = lds128(hpos + h);
            const float dx = (float)(int)(pi.x - q.x) * qs0, dy = (float)(int)(pi.y - q.y) * qs1,
                        dz = (float)(int)(pi.z - q.z) * qs2;
            const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, dx * dx));
            const long long j = adj_checked(b.ctl, (long long)q.w, b.S);
            if (!(r2 < lo) && r2 < hi && adj_r2_exact(b.x[b.ctl->cur], b.S, i, j, R.L) < R.rc2)
                hvp_pair2(make_float2(dx, 0.f), make_float2(dy, 0.f), make_float2(dz, 0.f),
                          make_float2(rcp_approx_f(r2), 0.f), __ldg(b.adj_wa + j), __ldg(b.adj_wb + j), z4, z2, wai,
                          wbi, sig2, eps24, isig, a);
        }
    }
}

__global__ void __launch_bounds__(kBlock, 4) k_adj_hvp32(Bufs b, const double *w, double *out, double scale,
                                                         double *acc)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Piece pc[kMaxPieces + 1];
    __shared__ Tile tl;
    __shared__ int s_tile, s_np, s_self;
    __shared__ double sm4[kBlock / 32][2];
    __shared__ __align__(8) unsigned long long s_mbar;   // completion of a tile's bulk copies
    __shared__ bool last;
    if (block_uniform(b.ctl->err != 0)) return;
    const int cur = b.ctl->cur;
    const uint4 *P = b.pos[cur];
    uint4 *hpos = reinterpret_cast<uint4 *>(smem_raw);
    unsigned short *lst = reinterpret_cast<unsigned short *>(smem_raw + (size_t)b.hcap * sizeof(uint4));
    if (threadIdx.x == 0) mbar_init(&s_mbar, 1);
    unsigned phase = 0;
    int err = 0;
    for (;;) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(&b.ctl->tile_next, 1u);
        __syncthreads();
        const int t = s_tile;
        if (t >= b.ctl->ntiles) break;
        load_tile(b, t, tl, pc, s_np);
        __syncthreads();
        const Replica &R = b.rep[tl.rep];
        const int np = s_np;
        const int Pt = tl.s1 - tl.s0;
        const int H = pc[np].hoff;
        double p0 = 0.0, p1 = 0.0;
        if (H <= b.hcap) {   // block-uniform; the list build rejects larger halos first
            if (threadIdx.x == 0) s_self = tile_self_offset(R, tl, pc, np);
            if (threadIdx.x < 32) issue_tile_bulk(b, tl, pc, np, P, hpos, lst, &s_mbar, threadIdx.x);
            const bool late = !mbar_wait(&s_mbar, phase);
            phase ^= 1u;
            if (__syncthreads_or(late)) {   // a bulk copy never completed: stop, report
                err |= kErrTimeout;
                break;
            }
            // the fourth word of each staged position becomes its slot
            stage_halo<uint4>(pc, np, [&](int h, int j) { hpos[h].w = (unsigned)j; });
            __syncthreads();
            const bool lstaged = tl.kmax * Pt <= kListStage * kTileMax;
            const double ieps = 1.0 / R.eps;
            for (long long i = tl.s0 + threadIdx.x; i < tl.s1; i += blockDim.x) {
                const int p = (int)(i - tl.s0);
                const uint4 pi = lds128(hpos + adj_checked(b.ctl, s_self + p, H));
                const int id = (int)adj_checked(b.ctl, (int)P[i].w, b.N);
                const int n = min(b.nn[i], b.K);
                const int npad = min(((n + kPad - 1) / kPad) * kPad, b.K);
                const float4 wai = b.adj_wa[i];
                const float2 wbi = b.adj_wb[i];
                HvpSums a;
                a.ax = a.ay = a.az = a.fx = a.fy = a.fz = a.sx = a.sy = a.sz = make_float2(0.f, 0.f);
                if (lstaged) hvp_particle<true>(b, R, hpos, H, lst + p, Pt, n, npad, pi, i, wai, wbi, a);
                else
                    hvp_particle<false>(b, R, hpos, H, b.nbr + nbr_index(tl.s0, Pt, b.K, 0, p), Pt, n, npad, pi, i,
                                        wai, wbi, a);
                out[id] = (double)(a.ax.x + a.ax.y);
                out[b.N + id] = (double)(a.ay.x + a.ay.y);
                out[2 * b.N + id] = (double)(a.az.x + a.az.y);
                const double wi0 = w[id], wi1 = w[b.N + id], wi2 = w[2 * b.N + id];
                p0 += (wi0 * (a.fx.x + a.fx.y) + wi1 * (a.fy.x + a.fy.y) + wi2 * (a.fz.x + a.fz.y)) * ieps;
                p1 += wi0 * (a.sx.x + a.sx.y) + wi1 * (a.sy.x + a.sy.y) + wi2 * (a.sz.x + a.sz.y);
            }
        } else {
            err |= kErrList;
        }
        // per-tile partials in a fixed order (zero for a rejected tile)
        for (int o = 16; o > 0; o >>= 1) {
            p0 += __shfl_down_sync(0xffffffffu, p0, o);
            p1 += __shfl_down_sync(0xffffffffu, p1, o);
        }
        if ((threadIdx.x & 31) == 0) { sm4[threadIdx.x >> 5][0] = p0; sm4[threadIdx.x >> 5][1] = p1; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0, c = 0;
            for (int q = 0; q < kBlock / 32; ++q) { a += sm4[q][0]; c += sm4[q][1]; }
            b.partial[4 * t + 0] = a;
            b.partial[4 * t + 1] = c;
            b.partial[4 * t + 2] = 0.0;
            b.partial[4 * t + 3] = 0.0;
        }
        __syncthreads();
    }
    if (err) atomicOr(&b.ctl->err, err);
    if (threadIdx.x == 0) {
        __threadfence();
        last = (atomicAdd(&b.ctl->done_force, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    adj_reduce(b, scale, acc);
    if (threadIdx.x == 0) {
        b.ctl->tile_next = 0u;
        b.ctl->done_force = 0u;
    }
}

// lx += c hv; then lv += dt lx (caller order, 3 N values each).
__global__ void k_adj_update(long long n3, double *lx, double *lv, const double *hv, double c, double dt)
{
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n3; q += (long long)gridDim.x * blockDim.x) {
        const double x = lx[q] + c * hv[q];
        lx[q] = x;
        lv[q] += dt * x;
    }
}

// Terminal adjoints of a loss on the final state itself: lx += dL/dx_T,
// lv += dL/dv_T (caller order, 3 N values each; either input may be null).
__global__ void k_adj_add(long long n3, double *lx, double *lv, const double *gx, const double *gv)
{
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n3; q += (long long)gridDim.x * blockDim.x) {
        if (gx) lx[q] += gx[q];
        if (gv) lv[q] += gv[q];
    }
}

// Explicit parameter terms of the loss from the per-replica sums (U, W, Ws):
// g_eps += (cU U + cW W) / eps, g_sigma += cU W / sigma + cW Ws (r_cut moves
// with sigma, so dU/dsigma = W / sigma); g holds (g_eps, g_sigma, -, -) per replica.
__global__ void k_adj_finish_loss(Bufs b, const double *sums, const double *coef, double *g)
{
    for (int r = 0; r < b.nrep; ++r) {
        const double U = sums[4 * r], W = sums[4 * r + 1], Ws = sums[4 * r + 2];
        const double cU = coef[4 * r], cW = coef[4 * r + 2];
        g[4 * r + 0] += (cU * U + cW * W) / b.rep[r].eps;
        g[4 * r + 1] += cU * W / b.rep[r].sigma + cW * Ws;
    }
}

static int adj_grid(const void *fn, size_t smem)
{
    int dev = 0, nsm = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kBlock, smem);
    return (occ > 0 ? occ : 1) * (nsm > 0 ? nsm : 1);
}

// hv = J w at the current state; g[4 r + k] += scale * (w.F/eps, w.dF/dsigma)_r.
// precision 1: FP32 pair terms (k_adj_hvp32), else FP64.
void launch_adj_hvp(const Bufs &b, int precision, const double *w, double *hv, double scale, double *g,
                    cudaStream_t st)
{
    if (precision == 1) {
        const size_t smem32 = (size_t)b.hcap * sizeof(uint4) + (size_t)kListStage * kTileMax * sizeof(unsigned short);
        static int grid32 = 0;
        static size_t gs32 = 0;
        if (grid32 == 0 || gs32 != smem32) { grid32 = adj_grid((const void *)k_adj_hvp32, smem32); gs32 = smem32; }
        k_adj_wslots<<<(unsigned)((b.S + 255) / 256), 256, 0, st>>>(b, w);
        k_adj_hvp32<<<grid32, kBlock, smem32, st>>>(b, w, hv, scale, g);
        return;
    }
    const size_t smem = (size_t)b.hcap * 6 * sizeof(double);
    static int grid = 0;
    static size_t gs = 0;
    if (grid == 0 || gs != smem) { grid = adj_grid((const void *)k_adj<0>, smem); gs = smem; }
    k_adj<0><<<grid, kBlock, smem, st>>>(b, w, hv, nullptr, nullptr, scale, g);
}

// lx, lv of the loss at the current state; sums[4 r + k] += (U, W, Ws)_r.
void launch_adj_loss(const Bufs &b, const double *coef, double *lx, double *lv, double *sums, cudaStream_t st)
{
    const size_t smem = (size_t)b.hcap * 6 * sizeof(double);
    static int grid = 0;
    static size_t gs = 0;
    if (grid == 0 || gs != smem) { grid = adj_grid((const void *)k_adj<1>, smem); gs = smem; }
    k_adj<1><<<grid, kBlock, smem, st>>>(b, nullptr, lx, lv, coef, 1.0, sums);
}

void launch_adj_finish_loss(const Bufs &b, const double *sums, const double *coef, double *g, cudaStream_t st)
{
    k_adj_finish_loss<<<1, 1, 0, st>>>(b, sums, coef, g);
}

void launch_adj_update(long long n3, double *lx, double *lv, const double *hv, double c, double dt, cudaStream_t st)
{
    k_adj_update<<<(unsigned)std::min<long long>((n3 + 255) / 256, 4096), 256, 0, st>>>(n3, lx, lv, hv, c, dt);
}

void launch_adj_add(long long n3, double *lx, double *lv, const double *gx, const double *gv, cudaStream_t st)
{
    k_adj_add<<<(unsigned)std::min<long long>((n3 + 255) / 256, 4096), 256, 0, st>>>(n3, lx, lv, gx, gv);
}

}  // namespace mdk
