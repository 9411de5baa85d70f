// Force evaluation that allocates no memory, for callers that cannot call
// cudaMalloc: a host framework that owns every byte of device memory through
// its own pool and forbids other allocators, or a process whose device
// memory is already committed to a fixed budget.  The caller passes device
// inputs and outputs; the only scratch, the per-block energy partials, lives
// in a file-scope device array that every GPU loading this library holds
// until the process exits.
//
// The pair arithmetic is the library's non-bonded term (shifted LJ / WCA
// under r < r_cut, minimum image, FP32 pairs with 64-bit fixed-point sums or
// FP64), summed directly over all pairs, without cells or Verlet lists:
// O(N^2), meant for systems of up to kNoAllocMaxN particles.  Bonded terms
// (FENE, angles) are not evaluated here.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "md.h"

namespace {

constexpr int kThreads = 128;
constexpr int kMaxBlocks = 4096;
constexpr long long kNoAllocMaxN = (long long)kThreads * kMaxBlocks;   // 524,288 particles

// Scratch shared by every call on a device: kMaxBlocks x (U, W) partials.
// Each call overwrites the partials of the blocks it launches before reading
// them, so nothing needs clearing; calls that overlap on the GPU race on it.
static __device__ __align__(256) double g_noalloc_partials[kMaxBlocks * 2];

constexpr float kMagic = 12582912.0f;   // 1.5 * 2^23
constexpr unsigned kMagicBits = 0x4B400000u;

__device__ __forceinline__ void fix_add(float a, float c, unsigned &hi, unsigned &lo)
{
    const float t1 = __fmaf_rn(a, c, kMagic);
    const float h = __fsub_rn(t1, kMagic);
    const float r = __fmaf_rn(a, c, -h);
    const float t2 = __fmaf_rn(r, 4194304.0f, kMagic);
    hi += __float_as_uint(t1) - kMagicBits;
    lo += __float_as_uint(t2) - kMagicBits;
}

__device__ __forceinline__ double fix_value(unsigned hi, unsigned lo)
{
    return (double)((long long)(int)hi * 4194304LL + (long long)(int)lo) * (1.0 / 4194304.0);
}

struct DirectParams {
    long long n;
    double L[3], to_q[3];
    float qs[3];
    double eps, sigma, rc2, vshift;
    float eps24_f, eps4_f, sig2_f, vshift_f, rc2_lo, rc2_hi;
    float fmax2;   // FP32: smallest r^2 at which a pair-force component stays inside the fixed-point range
};

__device__ __noinline__ double r2_exact(const double *x, long long n, long long i, long long j, const double *L)
{
    double d[3];
    for (int k = 0; k < 3; ++k) {
        const double t = __dsub_rn(x[k * n + i], x[k * n + j]);
        const double q = rint(__ddiv_rn(t, L[k]));
        d[k] = __dsub_rn(t, __dmul_rn(L[k], q));
    }
    return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

// One thread per particle i, all j in blocks staged through shared memory.
template <int PREC>
__global__ void __launch_bounds__(kThreads) k_direct(DirectParams p, const double *x, double *f, double *partials)
{
    __shared__ double sx[kThreads], sy[kThreads], sz[kThreads];
    __shared__ double red[kThreads][2];
    const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
    const bool real = i < p.n;
    const double xi = real ? x[i] : 0.0, yi = real ? x[p.n + i] : 0.0, zi = real ? x[2 * p.n + i] : 0.0;
    unsigned hx = 0, lx = 0, hy = 0, ly = 0, hz = 0, lz = 0, hu = 0, lu = 0, hw = 0, lw = 0;
    double F[3] = {0.0, 0.0, 0.0}, U = 0.0, W = 0.0;
    unsigned qi[3] = {0u, 0u, 0u};
    bool tooclose = false;   // FP32: a pair closer than the fixed-point range allows (or coincident)
    if (PREC == 1 && real) {
        const double xyz[3] = {xi, yi, zi};
        for (int k = 0; k < 3; ++k) qi[k] = (unsigned)(__double2ll_rn(xyz[k] * p.to_q[k]) & 0xffffffffLL);
    }
    for (long long j0 = 0; j0 < p.n; j0 += kThreads) {
        __syncthreads();
        const long long jl = j0 + threadIdx.x;
        if (jl < p.n) { sx[threadIdx.x] = x[jl]; sy[threadIdx.x] = x[p.n + jl]; sz[threadIdx.x] = x[2 * p.n + jl]; }
        __syncthreads();
        const int m = (int)min((long long)kThreads, p.n - j0);
        if (!real) continue;
        for (int u = 0; u < m; ++u) {
            const long long j = j0 + u;
            if (j == i) continue;
            if (PREC == 1) {
                const unsigned qj0 = (unsigned)(__double2ll_rn(sx[u] * p.to_q[0]) & 0xffffffffLL);
                const unsigned qj1 = (unsigned)(__double2ll_rn(sy[u] * p.to_q[1]) & 0xffffffffLL);
                const unsigned qj2 = (unsigned)(__double2ll_rn(sz[u] * p.to_q[2]) & 0xffffffffLL);
                const float dx = (float)(int)(qi[0] - qj0) * p.qs[0];
                const float dy = (float)(int)(qi[1] - qj1) * p.qs[1];
                const float dz = (float)(int)(qi[2] - qj2) * p.qs[2];
                const float r2 = dx * dx + dy * dy + dz * dz;
                if (!(r2 < p.rc2_hi)) continue;
                if (!(r2 < p.rc2_lo) && !(r2_exact(x, p.n, i, j, p.L) < p.rc2)) continue;
                // the two-integer split is exact only for |f d| < 2^21: such a
                // pair (and r = 0) poisons this particle's results instead
                if (r2 < p.fmax2) { tooclose = true; continue; }
                const float ir2 = 1.0f / r2;
                const float s2 = p.sig2_f * ir2, s6 = s2 * s2 * s2;
                const float fs = p.eps24_f * s6 * (2.0f * s6 - 1.0f) * ir2;
                fix_add(fs, dx, hx, lx);
                fix_add(fs, dy, hy, ly);
                fix_add(fs, dz, hz, lz);
                fix_add(p.eps4_f * s6 * (s6 - 1.0f) - p.vshift_f, 1.0f, hu, lu);
                fix_add(fs, r2, hw, lw);
            } else {
                double d[3] = {xi - sx[u], yi - sy[u], zi - sz[u]};
                for (int k = 0; k < 3; ++k) d[k] -= p.L[k] * rint(d[k] / p.L[k]);
                const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (!(r2 < p.rc2 * (1.0 + 1e-12))) continue;
                if (!(r2 < p.rc2 * (1.0 - 1e-12)) && !(r2_exact(x, p.n, i, j, p.L) < p.rc2)) continue;
                const double ir2 = 1.0 / r2, s2 = p.sigma * p.sigma * ir2, s6 = s2 * s2 * s2;
                const double fs = 24.0 * p.eps * s6 * (2.0 * s6 - 1.0) * ir2;
                for (int k = 0; k < 3; ++k) F[k] += fs * d[k];
                U += 4.0 * p.eps * s6 * (s6 - 1.0) - p.vshift;
                W += fs * r2;
            }
        }
    }
    if (PREC == 1) {
        F[0] = fix_value(hx, lx);
        F[1] = fix_value(hy, ly);
        F[2] = fix_value(hz, lz);
        U = fix_value(hu, lu);
        W = fix_value(hw, lw);
        if (tooclose) {
            const double qnan = __longlong_as_double(0x7ff8000000000000LL);
            F[0] = F[1] = F[2] = U = W = qnan;
        }
    }
    if (real)
        for (int k = 0; k < 3; ++k) f[k * p.n + i] = F[k];
    // half of each pair's energy and virial belongs to each end
    red[threadIdx.x][0] = real ? 0.5 * U : 0.0;
    red[threadIdx.x][1] = real ? 0.5 * W : 0.0;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            red[threadIdx.x][0] += red[threadIdx.x + s][0];
            red[threadIdx.x][1] += red[threadIdx.x + s][1];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x + 0] = red[0][0];
        partials[2 * blockIdx.x + 1] = red[0][1];
    }
}

// Sum the block partials in a fixed order and the kinetic energy; one block.
__global__ void __launch_bounds__(kThreads) k_direct_sum(long long n, int nblk, const double *partials,
                                                         const double *v, double mass, double *euw)
{
    __shared__ double red[kThreads][3];
    double U = 0.0, W = 0.0, K = 0.0;
    for (int q = threadIdx.x; q < nblk; q += kThreads) { U += partials[2 * q]; W += partials[2 * q + 1]; }
    if (v)
        for (long long i = threadIdx.x; i < n; i += kThreads)
            for (int k = 0; k < 3; ++k) K += 0.5 * mass * v[k * n + i] * v[k * n + i];
    red[threadIdx.x][0] = U; red[threadIdx.x][1] = K; red[threadIdx.x][2] = W;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int k = 0; k < 3; ++k) red[threadIdx.x][k] += red[threadIdx.x + s][k];
        __syncthreads();
    }
    if (threadIdx.x == 0) { euw[0] = red[0][0]; euw[1] = red[0][1]; euw[2] = red[0][2]; }
}

// Device address of the scratch array, looked up once per device with that
// device current (in host code the array's name is only a host-side stand-in)
// and kept for the life of the process: a cudaDeviceReset, which ends the
// device's primary context, leaves a stale address behind.
std::mutex g_mutex;
double *g_scratch_ptr[64] = {nullptr};

cudaError_t scratch_for_current_device(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

void set_msg(char *msg, int len, const char *text)
{
    if (msg && len > 0) {
        std::strncpy(msg, text, (size_t)len - 1);
        msg[len - 1] = '\0';
    }
}

}  // namespace

extern "C" md_status md_compute_forces_noalloc(const double *x, const double *v, int64_t n, const double *box,
                                               double eps, double sigma, double rc, int32_t shift,
                                               int32_t precision, double mass, double *f_out, double *euw_out,
                                               char *err_msg, int32_t err_len, void *stream)
{
    set_msg(err_msg, err_len, "");
    if (n < 1 || n > kNoAllocMaxN) {
        char t[160];
        std::snprintf(t, sizeof t, "md_compute_forces_noalloc: n = %lld outside [1, %lld] (fixed scratch size)",
                      (long long)n, (long long)kNoAllocMaxN);
        set_msg(err_msg, err_len, t);
        return MD_ERR_ARG;
    }
    if (!x || !f_out || !box || !(eps > 0) || !(sigma > 0) || !(rc > 0) || !(mass > 0) ||
        (precision != MD_FP64 && precision != MD_FP32_FIXED)) {
        set_msg(err_msg, err_len, "md_compute_forces_noalloc: bad argument");
        return MD_ERR_ARG;
    }
    DirectParams p{};
    p.n = n;
    for (int k = 0; k < 3; ++k) {
        if (!(box[k] >= 2.0 * rc)) {
            set_msg(err_msg, err_len, "md_compute_forces_noalloc: box edge shorter than 2 r_cut");
            return MD_ERR_BOX_TOO_SMALL;
        }
        p.L[k] = box[k];
        p.to_q[k] = 4294967296.0 / box[k];
        p.qs[k] = (float)(box[k] / 4294967296.0);
    }
    const double s6 = std::pow(sigma / rc, 6.0);
    p.eps = eps;
    p.sigma = sigma;
    p.rc2 = rc * rc;
    p.vshift = shift ? 4.0 * eps * (s6 * s6 - s6) : 0.0;
    p.eps24_f = (float)(24.0 * eps);
    p.eps4_f = (float)(4.0 * eps);
    p.sig2_f = (float)(sigma * sigma);
    p.vshift_f = (float)p.vshift;
    double Lmax = std::fmax(box[0], std::fmax(box[1], box[2]));
    const double band = 2.0 * rc * std::sqrt(3.0) * Lmax / 4294967296.0 + std::ldexp(1.0, -16) * rc * rc;
    p.rc2_lo = (float)(rc * rc - band);
    p.rc2_hi = (float)(rc * rc + band);
    {
        // smallest r at which the pair force 24 eps (2 (s/r)^12 - (s/r)^6) / r
        // stays below 0.9 x 2^21, by bisection (the force falls with r there)
        double lo = 1e-3 * sigma, hi = rc;
        for (int it = 0; it < 200; ++it) {
            const double mid = 0.5 * (lo + hi);
            const double m6 = std::pow(sigma / mid, 6.0);
            const double fm = 24.0 * eps * (2.0 * m6 * m6 - m6) / mid;
            if (fm > std::ldexp(1.0, 21) * 0.9) lo = mid; else hi = mid;
        }
        p.fmax2 = (float)(hi * hi);
    }
    double *scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) {
        set_msg(err_msg, err_len, cudaGetErrorString(e));
        return MD_ERR_CUDA;
    }
    const int nblk = (int)((n + kThreads - 1) / kThreads);
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == MD_FP32_FIXED) k_direct<1><<<nblk, kThreads, 0, st>>>(p, x, f_out, scratch);
    else k_direct<0><<<nblk, kThreads, 0, st>>>(p, x, f_out, scratch);
    if (euw_out) k_direct_sum<<<1, kThreads, 0, st>>>(n, nblk, scratch, v, mass, euw_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_msg(err_msg, err_len, cudaGetErrorString(e));
        return MD_ERR_CUDA;
    }
    return MD_OK;
}
