// bd_static.cu -- bdecon_log_posterior_static: the log posterior of Eq. 9
// for an object given in device memory, evaluated without allocating any
// device memory.  All scratch lives in one file-scope __device__ array.
//
// Who needs this: programs that must not call cudaMalloc / cudaFree at all
// once they are running -- for example an acquisition loop that reserved all
// device memory for frame buffers up front, or a host whose allocator is
// owned by another framework and forbids outside allocations (and the
// device synchronisation cudaMalloc/cudaFree can cause) -- can still score a
// candidate object.  The regular path (bdecon_log_posterior) needs a handle,
// and creating a handle allocates.
#include <cstdio>
#include <mutex>

#include "bdecon.h"
#include "bd_device.cuh"

namespace bd {

// Static scratch: 2^19 doubles (4 MiB), held by every GPU that loads the
// library until the process exits.
constexpr int64_t kStaticDoubles = int64_t(1) << 19;
static __device__ __align__(256) double g_static_scratch[kStaticDoubles];

constexpr int kMaxDevices = 64;
static double* g_scratch_addr[kMaxDevices];
static std::mutex g_scratch_mu;

namespace {

struct StaticArgs {
    int H, W, L, R, S, Ho, Wo, npi, npj;
    const float *w, *g, *o, *v;
    double gs, os, vs;
    const double* psf;
    const double* rho;
    double* K;          // scratch L*L
    double* alpha;      // scratch 4 * S*S (one block per patch shape)
    double* kw;         // scratch S*S
    double* part_ll;    // scratch nblk
    double* part_lp;    // scratch npi*npj
};

__device__ __forceinline__ double sblock_sum(double v, double* sh)
{
    const int tid = threadIdx.x;
    sh[tid] = v;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
        if (tid < o) sh[tid] += sh[tid + o];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ void shape_sides(const StaticArgs& a, int s, int* ph, int* pw)
{
    const int rh = a.Ho - (a.npi - 1) * a.S, rw = a.Wo - (a.npj - 1) * a.S;
    *ph = (s & 2) ? rh : a.S;
    *pw = (s & 1) ? rw : a.S;
}

// normalised PSF and the Eq. 8 hyperparameter of every patch shape
__global__ void __launch_bounds__(kRedThreads) k_static_alpha(StaticArgs a)
{
    __shared__ double sh[kRedThreads];
    __shared__ double2 eh[kMaxS], ew[kMaxS];
    double s = 0.0;
    for (int k = threadIdx.x; k < a.L * a.L; k += kRedThreads) s += a.psf[k];
    const double tot = sblock_sum(s, sh);
    for (int k = threadIdx.x; k < a.L * a.L; k += kRedThreads) a.K[k] = a.psf[k] / tot;
    __syncthreads();
    for (int sidx = 0; sidx < kMaxShapes; ++sidx) {
        int ph, pw;
        shape_sides(a, sidx, &ph, &pw);
        const int n = ph * pw;
        // the previous call's contents are still in the array: clear before accumulating
        for (int k = threadIdx.x; k < n; k += kRedThreads) a.kw[k] = 0.0;
        __syncthreads();
        if (threadIdx.x == 0)
            for (int p = 0; p < a.L; ++p)
                for (int q = 0; q < a.L; ++q) {
                    const int x = ((p - a.R) % ph + ph) % ph, y = ((q - a.R) % pw + pw) % pw;
                    a.kw[x * pw + y] += a.K[p * a.L + q];
                }
        // twiddles exp(-2 pi i j / ph) and exp(-2 pi i j / pw), as in k_static_prior
        for (int j = threadIdx.x; j < ph; j += kRedThreads) {
            double sn, cs;
            sincospi(2.0 * (double)j / ph, &sn, &cs);
            eh[j] = make_double2(cs, -sn);
        }
        for (int j = threadIdx.x; j < pw; j += kRedThreads) {
            double sn, cs;
            sincospi(2.0 * (double)j / pw, &sn, &cs);
            ew[j] = make_double2(cs, -sn);
        }
        __syncthreads();
        double part = 0.0;
        double* al = a.alpha + (size_t)sidx * a.S * a.S;
        for (int idx = threadIdx.x; idx < n; idx += kRedThreads) {
            const int k = idx / pw, l = idx % pw;
            double re = 0.0, im = 0.0;
            for (int u = 0; u < ph; ++u) {
                const double2 e1 = eh[(k * u) % ph];
                for (int v = 0; v < pw; ++v) {
                    const double2 e2 = ew[(l * v) % pw];
                    const double x = a.kw[u * pw + v];
                    re += x * (e1.x * e2.x - e1.y * e2.y);
                    im += x * (e1.x * e2.y + e1.y * e2.x);
                }
            }
            al[idx] = hypot(re, im);
            part += al[idx];
        }
        __syncthreads();
        const double tsum = sblock_sum(part, sh);
        for (int idx = threadIdx.x; idx < n; idx += kRedThreads) al[idx] /= tsum;
        __syncthreads();
    }
}

// expected image (Eq. 1-2) and per-pixel log likelihood (Eq. 6), block partials
__global__ void __launch_bounds__(kRedThreads) k_static_lik(StaticArgs a)
{
    __shared__ double sh[kRedThreads];
    const int idx = blockIdx.x * kRedThreads + threadIdx.x;
    double ll = 0.0;
    if (idx < a.H * a.W) {
        const int r = idx / a.W, c = idx % a.W;
        double mu = 0.0;
        for (int p = 0; p < a.L; ++p) {
            const double* row = a.rho + (size_t)(r + 2 * a.R - p) * a.Wo + (c + 2 * a.R);
            for (int q = 0; q < a.L; ++q) mu += a.K[p * a.L + q] * row[-q];
        }
        const double G = a.g ? (double)a.g[idx] : a.gs;
        const double off = a.o ? (double)a.o[idx] : a.os;
        const double var = a.v ? (double)a.v[idx] : a.vs;
        const double is2 = G * G / var;
        ll = loglik64(mu, ((double)a.w[idx] - off) / G, is2, exp(-is2), -0.5 * log(2.0 * CUDART_PI * var));
    }
    const double s = sblock_sum(ll, sh);
    if (threadIdx.x == 0) a.part_ll[blockIdx.x] = s;
}

// patch log prior (Eq. 7-8) over all ph*pw frequencies, one block per patch
__global__ void __launch_bounds__(kRedThreads) k_static_prior(StaticArgs a)
{
    __shared__ double sh[kRedThreads];
    __shared__ double2 eh[kMaxS], ew[kMaxS];
    const int p = blockIdx.x, pi = p / a.npj, pj = p % a.npj;
    const int sidx = (((pi + 1) * a.S > a.Ho) ? 2 : 0) | (((pj + 1) * a.S > a.Wo) ? 1 : 0);
    int ph, pw;
    shape_sides(a, sidx, &ph, &pw);
    for (int j = threadIdx.x; j < ph; j += kRedThreads) {
        double sn, cs;
        sincospi(2.0 * (double)j / ph, &sn, &cs);
        eh[j] = make_double2(cs, -sn);
    }
    for (int j = threadIdx.x; j < pw; j += kRedThreads) {
        double sn, cs;
        sincospi(2.0 * (double)j / pw, &sn, &cs);
        ew[j] = make_double2(cs, -sn);
    }
    __syncthreads();
    const double* rho = a.rho + (size_t)pi * a.S * a.Wo + pj * a.S;
    const double* al = a.alpha + (size_t)sidx * a.S * a.S;
    double sl = 0.0, sm = 0.0;
    for (int idx = threadIdx.x; idx < ph * pw; idx += kRedThreads) {
        const int k = idx / pw, l = idx % pw;
        double re = 0.0, im = 0.0;
        for (int u = 0; u < ph; ++u) {
            const double2 e1 = eh[(k * u) % ph];
            for (int v = 0; v < pw; ++v) {
                const double2 e2 = ew[(l * v) % pw];
                const double x = rho[(size_t)u * a.Wo + v];
                re += x * (e1.x * e2.x - e1.y * e2.y);
                im += x * (e1.x * e2.y + e1.y * e2.x);
            }
        }
        const double m = sqrt(re * re + im * im);
        sl += (al[idx] - 1.0) * log(m);
        sm += m;
    }
    const double tl = sblock_sum(sl, sh);
    const double tm = sblock_sum(sm, sh);
    if (threadIdx.x == 0) a.part_lp[p] = tl + (double)(ph * pw - 1) * log(tm);
}

__global__ void __launch_bounds__(kRedThreads) k_static_total(const double* pll, int nll, const double* plp, int nlp,
                                                             double* out)
{
    __shared__ double sh[kRedThreads];
    double x = 0.0, y = 0.0;
    for (int k = threadIdx.x; k < nll; k += kRedThreads) x += pll[k];
    for (int k = threadIdx.x; k < nlp; k += kRedThreads) y += plp[k];
    const double tx = sblock_sum(x, sh);
    const double ty = sblock_sum(y, sh);
    if (threadIdx.x == 0) out[0] = tx + ty;
}

bdecon_status sfail(bdecon_status s, const char* msg)
{
    set_host_error(msg);   // readable through bdecon_last_error(NULL)
    return s;
}

}  // namespace

// Device address of the static scratch on the current device.  Host code must
// not pass g_static_scratch itself to a kernel: in host code that name is a
// host-side stand-in, not a device address.  Looked up once per device.
static bdecon_status static_scratch(double** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return sfail(BDECON_ERR_CUDA, "no current CUDA device");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) return sfail(BDECON_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
        g_scratch_addr[dev] = (double*)p;
    }
    *out = g_scratch_addr[dev];
    return BDECON_OK;
}

}  // namespace bd

extern "C" bdecon_status bdecon_log_posterior_static(int32_t H, int32_t W, const float* image, int32_t L,
                                                     const double* psf, const float* gain_map, double gain,
                                                     const float* offset_map, double offset, const float* var_map,
                                                     double read_var, int32_t stride, const double* rho, double* out,
                                                     void* stream)
{
    using namespace bd;
    if (H < 1 || W < 1 || L < 1 || L % 2 == 0 || L > kMaxL)
        return sfail(BDECON_ERR_INVALID, "frame size or PSF side out of range (L odd, 1..63)");
    const int S = stride ? stride : L;
    if (S < L || S > kMaxS) return sfail(BDECON_ERR_INVALID, "stride must be in [L, 64]");
    if (!image || !psf || !rho || !out) return sfail(BDECON_ERR_INVALID, "image, psf, rho and out are required");
    if ((!gain_map && !(gain > 0.0)) || (!var_map && !(read_var > 0.0)))
        return sfail(BDECON_ERR_INVALID, "scalar gain and read_var must be > 0");
    StaticArgs a;
    a.H = H; a.W = W; a.L = L; a.R = L / 2; a.S = S;
    a.Ho = H + 2 * a.R; a.Wo = W + 2 * a.R;
    a.npi = (a.Ho + S - 1) / S; a.npj = (a.Wo + S - 1) / S;
    a.w = image; a.g = gain_map; a.o = offset_map; a.v = var_map;
    a.gs = gain; a.os = offset; a.vs = read_var;
    a.psf = psf; a.rho = rho;
    const int64_t nblk = ((int64_t)H * W + kRedThreads - 1) / kRedThreads;
    const int64_t npatch = (int64_t)a.npi * a.npj;
    const int64_t need = (int64_t)L * L + 5 * (int64_t)S * S + nblk + npatch;
    if (need > kStaticDoubles) {
        char msg[200];
        snprintf(msg, sizeof msg, "problem needs %lld scratch doubles; the static scratch holds %lld",
                 (long long)need, (long long)kStaticDoubles);
        return sfail(BDECON_ERR_INVALID, msg);
    }
    double* base = nullptr;
    bdecon_status s = static_scratch(&base);
    if (s != BDECON_OK) return s;
    a.K = base;
    a.alpha = a.K + (size_t)L * L;
    a.kw = a.alpha + 4 * (size_t)S * S;
    a.part_ll = a.kw + (size_t)S * S;
    a.part_lp = a.part_ll + nblk;
    cudaStream_t st = (cudaStream_t)stream;
    k_static_alpha<<<1, kRedThreads, 0, st>>>(a);
    k_static_lik<<<(unsigned)nblk, kRedThreads, 0, st>>>(a);
    k_static_prior<<<(unsigned)npatch, kRedThreads, 0, st>>>(a);
    k_static_total<<<1, kRedThreads, 0, st>>>(a.part_ll, (int)nblk, a.part_lp, (int)npatch, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return sfail(BDECON_ERR_CUDA, cudaGetErrorString(e));
    return BDECON_OK;
}
