// bd_state.cu -- set-up, refresh and read-out kernels of libbdecon.
//
//   a1  set-up (double): normalised PSF (Eq. 1-2), per-pixel photon-unit
//       constants of Eq. 4-6, Dirichlet hyperparameters |OTF| / sum |OTF| of
//       Eq. 8 per patch shape, twiddle tables, initial object.
//   a8  refresh (double): mu = K (x) rho by direct summation, patch spectra
//       by direct DFT, and the full log posterior of Eq. 9; it replaces the
//       incrementally updated mu and spectra (drift correction) and rebases
//       the trace.
// Every reduction uses a fixed block size and a fixed tree, so results do
// not depend on the launch plan of the sweep kernel.
#include <cmath>

#include <atomic>
#include <mutex>

#include "bd_device.cuh"

namespace bd {

// deterministic block sum (kRedThreads threads)
__device__ __forceinline__ double block_sum(double v, double* sh)
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

// ------------------------------------------------------------------ a1 ---
__global__ void __launch_bounds__(kRedThreads) k_setup_psf(int L, const double* psf, double* K64, float* K32)
{
    __shared__ double sh[kRedThreads];
    double s = 0.0;
    for (int k = threadIdx.x; k < L * L; k += kRedThreads) s += psf[k];
    const double tot = block_sum(s, sh);
    for (int k = threadIdx.x; k < L * L; k += kRedThreads) {
        const double v = psf[k] / tot;
        K64[k] = v;
        K32[k] = (float)v;
    }
}

// Effective kernel of a lattice f times finer than the camera: a camera
// pixel sums the f x f cells of its area (the pixel integral of Eq. 1), so
// Ke[p][q] = sum_{u,v < f} K[p-u][q-v], side Le = L + f - 1.
__global__ void k_setup_eff(int L, int f, const double* K64, double* Ke64, float* Ke32)
{
    const int Le = L + f - 1;
    for (int idx = threadIdx.x; idx < Le * Le; idx += blockDim.x) {
        const int p = idx / Le, q = idx % Le;
        double s = 0.0;
        for (int u = 0; u < f; ++u)
            for (int v = 0; v < f; ++v) {
                const int pp = p - u, qq = q - v;
                if (pp >= 0 && pp < L && qq >= 0 && qq < L) s += K64[pp * L + qq];
            }
        Ke64[idx] = s;
        Ke32[idx] = (float)s;
    }
}

// c = (w - o)/G, s^2 = var/G^2 (photon units), 1/s^2, exp(-1/s^2), -log(2 pi var)/2
__global__ void __launch_bounds__(kRedThreads) k_setup_data(int n, const float* w, const float* g, const float* o,
                                                           const float* v, double gs, double os, double vs,
                                                           double* dat64, float* dat32, double* part_c)
{
    __shared__ double sh[kRedThreads];
    const int idx = blockIdx.x * kRedThreads + threadIdx.x;
    double c = 0.0;
    if (idx < n) {
        const double G = g ? (double)g[idx] : gs;
        const double off = o ? (double)o[idx] : os;
        const double var = v ? (double)v[idx] : vs;
        c = ((double)w[idx] - off) / G;
        const double is2 = G * G / var;
        const double beta = exp(-is2);
        const double lnorm = -0.5 * log(2.0 * CUDART_PI * var);
        dat64[4 * (size_t)idx + 0] = c;
        dat64[4 * (size_t)idx + 1] = is2;
        dat64[4 * (size_t)idx + 2] = beta;
        dat64[4 * (size_t)idx + 3] = lnorm;
        dat32[4 * (size_t)idx + 0] = (float)c;
        dat32[4 * (size_t)idx + 1] = (float)is2;
        dat32[4 * (size_t)idx + 2] = (float)beta;
        dat32[4 * (size_t)idx + 3] = (float)lnorm;
    }
    const double s = block_sum(c, sh);
    if (threadIdx.x == 0) part_c[blockIdx.x] = s;
}

// b0 = max(0.1, mean_n c_n)
__global__ void __launch_bounds__(kRedThreads) k_setup_b0(const double* part_c, int nblk, int npix, int f, double* b0)
{
    __shared__ double sh[kRedThreads];
    double s = 0.0;
    for (int k = threadIdx.x; k < nblk; k += kRedThreads) s += part_c[k];
    const double tot = block_sum(s, sh);
    if (threadIdx.x == 0) {
        const double m = tot / (double)npix;
        b0[0] = (m > 0.1 ? m : 0.1) / (double)(f * f);   // a camera pixel collects f^2 cells
    }
}

// exp(-2 pi i j / n) for j < n
__global__ void k_setup_tw(int n, double* tw64, float* tw32)
{
    for (int j = threadIdx.x + blockIdx.x * blockDim.x; j < n; j += blockDim.x * gridDim.x) {
        double s, c;
        sincospi(2.0 * (double)j / (double)n, &s, &c);
        tw64[2 * j] = c;
        tw64[2 * j + 1] = -s;
        tw32[2 * j] = (float)c;
        tw32[2 * j + 1] = (float)-s;
    }
}

// Eq. 8 hyperparameter for one patch shape: alpha = |DFT(PSF wrapped onto the
// ph x pw torus, centre at the origin)| / sum, then the weights of the
// canonical half-spectrum entries: mult * (alpha - 1) / 2 and mult.
__global__ void __launch_bounds__(kRedThreads) k_setup_alpha(int L, const double* K64, int ph, int pw,
                                                            const int* ent_kl, int nhalf, double* kw,
                                                            double* mag, double* wa64, double* m64,
                                                            float* wa32, float* m32, const double2* twh,
                                                            const double2* tww)
{
    __shared__ double sh[kRedThreads];
    const int R = L / 2, n = ph * pw;
    if (threadIdx.x == 0) {
        for (int k = 0; k < n; ++k) kw[k] = 0.0;
        for (int p = 0; p < L; ++p)
            for (int q = 0; q < L; ++q) {
                const int x = ((p - R) % ph + ph) % ph, y = ((q - R) % pw + pw) % pw;
                kw[x * pw + y] += K64[p * L + q];
            }
    }
    __syncthreads();
    double part = 0.0;
    for (int idx = threadIdx.x; idx < n; idx += kRedThreads) {
        const int k = idx / pw, l = idx % pw;
        // exp(-2 pi i (k u / ph + l v / pw)) from the twiddle tables of the two sides
        double re = 0.0, im = 0.0;
        for (int u = 0; u < ph; ++u) {
            const double2 eh = twh[(k * u) % ph];
            for (int v = 0; v < pw; ++v) {
                const double2 ew = tww[(l * v) % pw];
                const double x = kw[u * pw + v];
                re += x * (eh.x * ew.x - eh.y * ew.y);
                im += x * (eh.x * ew.y + eh.y * ew.x);
            }
        }
        mag[idx] = hypot(re, im);
        part += mag[idx];
    }
    // the sum over all frequencies, in a fixed order
    __syncthreads();
    const double tot = block_sum(part, sh);
    for (int e = threadIdx.x; e < nhalf; e += kRedThreads) {
        const int kl = ent_kl[e];
        const int k = kl >> 16, l = kl & 0xffff;
        const bool self = ((ph - k) % ph == k) && ((pw - l) % pw == l);
        const double mult = self ? 1.0 : 2.0;
        const double a = mag[k * pw + l] / tot;
        wa64[e] = 0.5 * mult * (a - 1.0);
        m64[e] = mult;
        wa32[e] = (float)wa64[e];
        m32[e] = (float)mult;
    }
}

// Initial object rho0_m = b0 exp(z_m / 10), z_m the Box-Muller normal of the
// Philox counter (m, 0, chain, 0): sweep index 0 is never a sampling sweep.
template <typename T>
__global__ void k_init_rho(int n, uint32_t seed_lo, uint32_t seed_hi, int chain, const double* b0, T* rho)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    const uint4 x = philox4x32_10(make_uint4((uint32_t)m, 0u, (uint32_t)chain, 0u), seed_lo, seed_hi);
    const double z = sqrt(-2.0 * log(uniform23<double>(x.x))) * cos(2.0 * CUDART_PI * uniform23<double>(x.y));
    rho[m] = (T)(b0[0] * exp(0.1 * z));
}

void launch_setup(const Image& im, const Image* d_im, const float* w, const float* g, const float* o,
                  const float* v, double gs, double os, double vs, const double* psf_raw, double* b0_out,
                  double* scratch, cudaStream_t st, int64_t* launches)
{
    (void)d_im;
    k_setup_psf<<<1, kRedThreads, 0, st>>>(im.L, psf_raw, const_cast<double*>(im.K64), const_cast<float*>(im.K32));
    if (im.f > 1) {
        k_setup_eff<<<1, 256, 0, st>>>(im.L, im.f, im.K64, const_cast<double*>(im.Ke64), const_cast<float*>(im.Ke32));
        ++*launches;
    }
    const int npix = im.H * im.W;
    const int nblk = (npix + kRedThreads - 1) / kRedThreads;
    double* part_c = scratch;                       // nblk
    k_setup_data<<<nblk, kRedThreads, 0, st>>>(npix, w, g, o, v, gs, os, vs, const_cast<double*>(im.dat64),
                                               const_cast<float*>(im.dat32), part_c);
    k_setup_b0<<<1, kRedThreads, 0, st>>>(part_c, nblk, npix, im.f, b0_out);
    *launches += 3;
    // twiddles: the distinct patch sides appear at the shapes' offsets
    for (int s = 0; s < kMaxShapes; ++s) {
        const Shape& sh = im.shape[s];
        if (sh.nhalf == 0) continue;
        k_setup_tw<<<1, 128, 0, st>>>(sh.ph, const_cast<double*>(im.tw64) + 2 * sh.twh_off,
                                      const_cast<float*>(im.tw32) + 2 * sh.twh_off);
        k_setup_tw<<<1, 128, 0, st>>>(sh.pw, const_cast<double*>(im.tw64) + 2 * sh.tww_off,
                                      const_cast<float*>(im.tw32) + 2 * sh.tww_off);
        double* kw = scratch + nblk + 8;
        double* mag = kw + kMaxS * kMaxS;
        k_setup_alpha<<<1, kRedThreads, 0, st>>>(im.L, im.K64, sh.ph, sh.pw, im.ent_kl + sh.ent_off, sh.nhalf, kw,
                                                 mag, const_cast<double*>(im.ent_wa64) + sh.ent_off,
                                                 const_cast<double*>(im.ent_m64) + sh.ent_off,
                                                 const_cast<float*>(im.ent_wa32) + sh.ent_off,
                                                 const_cast<float*>(im.ent_m32) + sh.ent_off,
                                                 reinterpret_cast<const double2*>(im.tw64) + sh.twh_off,
                                                 reinterpret_cast<const double2*>(im.tw64) + sh.tww_off);
        *launches += 3;
    }
}

template <typename T>
void launch_init_rho(const Image& im, const Chain& ch, const double* b0, cudaStream_t st, int64_t* launches)
{
    const int n = im.Ho * im.Wo;
    k_init_rho<T><<<(n + 255) / 256, 256, 0, st>>>(n, im.seed_lo, im.seed_hi, ch.chain, b0, reinterpret_cast<T*>(ch.rho));
    ++*launches;
}
template void launch_init_rho<float>(const Image&, const Chain&, const double*, cudaStream_t, int64_t*);
template void launch_init_rho<double>(const Image&, const Chain&, const double*, cudaStream_t, int64_t*);

// ------------------------------------------------------------------ a8 ---
// mu = K (x) rho (Eq. 1-2) and the per-pixel log likelihood (Eq. 6), double.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_refresh_mu(Image im, Chain ch, double* part_ll, int write,
                                                           int* err)
{
    __shared__ double sh[kRedThreads];
    const int idx = blockIdx.x * kRedThreads + threadIdx.x;
    double ll = 0.0;
    if (idx < im.H * im.W) {
        const int a = idx / im.W, b = idx % im.W;
        const T* rho = reinterpret_cast<const T*>(ch.rho);
        // Eq. 1 on the object lattice: mu[a][b] = sum Ke[p][q] rho[f a + Le-1-p][f b + Le-1-q]
        const int Le = im.Le, f = im.f;
        double mu = 0.0;
        for (int p = 0; p < Le; ++p) {
            const T* row = rho + (size_t)(f * a + Le - 1 - p) * im.Wo + (f * b + Le - 1);
            for (int q = 0; q < Le; ++q) mu += im.Ke64[p * Le + q] * (double)row[-q];
        }
        if (!(mu > 0.0) || !isfinite(mu)) {
            atomicOr(err, kErrNumeric);
        } else {
            const double* d = im.dat64 + 4 * (size_t)idx;
            if (write && ch.phi) {   // augmented chain: the completed likelihood at its counts
                const int phi = (int)reinterpret_cast<const T*>(ch.phi)[(size_t)a * im.mu_pitch + b];
                ll = d[3] + phi_logterm(phi, ::log((double)(T)mu), d[0], d[1]) - (double)(T)mu;
            } else {
                ll = loglik64(mu, d[0], d[1], d[2], d[3]);
            }
            if (write && ch.cum) {
                // the cache describes the stored (rounded) expected image
                const Cum6 q = photon_cumulants<double>((double)(T)mu, d[0], d[1], d[2]);
                ch.cum[(size_t)a * im.mu_pitch + b] = q.a;
                ch.cum2[(size_t)a * im.mu_pitch + b] = q.b;
            }
        }
        if (write) reinterpret_cast<T*>(ch.mu)[(size_t)a * im.mu_pitch + b] = (T)mu;
    }
    const double s = block_sum(ll, sh);
    if (threadIdx.x == 0) part_ll[blockIdx.x] = s;
}

// Patch spectra by direct DFT (canonical half) and the patch log prior of Eq. 8:
//   sum_e mult_e (alpha_e - 1) log|X_e| + (K - 1) log sum_e mult_e |X_e|.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_refresh_spec(Image im, Chain ch, double* part_lp, int write)
{
    // one block per patch: its half spectrum by the 2-D DFT taken as two
    // 1-D transforms (rows, then columns), O(ph pw (ph + pw)) instead of
    // O((ph pw)^2) for the direct sum, in double in shared memory:
    //   Y[u][l] = sum_v x[u][v] exp(-2 pi i l v / pw),
    //   X[k][l] = sum_u Y[u][l] exp(-2 pi i k u / ph)
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ double sh[kRedThreads];
    const int p = blockIdx.x;
    const int pi = p / im.npj, pj = p % im.npj;
    const Shape& sp = im.shape[shape_index(im, pi, pj)];
    const int ph = sp.ph, pw = sp.pw, n = ph * pw;
    double* x = reinterpret_cast<double*>(dyn);                    // [ph][pw]
    double2* Y = reinterpret_cast<double2*>(dyn) + (n + 1) / 2;     // [ph][pw]
    const T* rho = reinterpret_cast<const T*>(ch.rho) + (size_t)pi * im.S * im.Wo + pj * im.S;
    const double2* twh = reinterpret_cast<const double2*>(im.tw64) + sp.twh_off;
    const double2* tww = reinterpret_cast<const double2*>(im.tw64) + sp.tww_off;
    for (int e = threadIdx.x; e < n; e += kRedThreads) {
        const int u = e / pw, v = e - (e / pw) * pw;
        x[e] = (double)rho[(size_t)u * im.Wo + v];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += kRedThreads) {
        const int u = e / pw, l = e - (e / pw) * pw;
        double re = 0.0, imv = 0.0;
        for (int v = 0; v < pw; ++v) {
            const double2 w = tww[(l * v) % pw];
            re += x[u * pw + v] * w.x;
            imv += x[u * pw + v] * w.y;
        }
        Y[e] = make_double2(re, imv);
    }
    __syncthreads();
    using T2 = typename Vec2<T>::type;
    T2* spec = reinterpret_cast<T2*>(ch.spec) + im.patch_off[p];
    double sl = 0.0, sm = 0.0;
    for (int e = threadIdx.x; e < sp.nhalf; e += kRedThreads) {
        const int kl = im.ent_kl[sp.ent_off + e];
        const int k = kl >> 16, l = kl & 0xffff;
        double re = 0.0, imv = 0.0;
        for (int u = 0; u < ph; ++u) {
            const double2 w = twh[(k * u) % ph];
            const double2 y = Y[u * pw + l];
            re += y.x * w.x - y.y * w.y;
            imv += y.x * w.y + y.y * w.x;
        }
        if (write) {
            T2 X;
            X.x = (T)re;
            X.y = (T)imv;
            spec[e] = X;
        }
        const double n2 = re * re + imv * imv;
        sl += im.ent_wa64[sp.ent_off + e] * log(n2);
        sm += im.ent_m64[sp.ent_off + e] * sqrt(n2);
    }
    const double tl = block_sum(sl, sh);
    const double tm = block_sum(sm, sh);
    if (threadIdx.x == 0) part_lp[p] = tl + (double)(sp.K - 1) * log(tm);
}

__global__ void __launch_bounds__(kRedThreads) k_refresh_total(const double* part_ll, int n_ll, const double* part_lp,
                                                              int n_lp, double* out, const int* out_index)
{
    __shared__ double sh[kRedThreads];
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < n_ll; k += kRedThreads) a += part_ll[k];
    for (int k = threadIdx.x; k < n_lp; k += kRedThreads) b += part_lp[k];
    const double ta = block_sum(a, sh);
    const double tb = block_sum(b, sh);
    if (threadIdx.x == 0) out[out_index ? *out_index : 0] = ta + tb;
}

template <typename T>
void launch_refresh(const Image& im, const Chain& ch, double* scratch, int write_state, double* out_logpost,
                    const int* out_index, int* err, cudaStream_t st, int64_t* launches)
{
    const int nblk = (im.H * im.W + kRedThreads - 1) / kRedThreads;
    double* part_ll = scratch;
    double* part_lp = scratch + nblk;
    k_refresh_mu<T><<<nblk, kRedThreads, 0, st>>>(im, ch, part_ll, write_state, err);
    // the patch and its row transforms in shared memory (24 bytes per patch pixel)
    const size_t smem = 8 * (size_t)(((size_t)im.S * im.S + 1) / 2 * 2) + 16 * (size_t)im.S * im.S;
    static std::atomic<size_t> limit{48 * 1024};   // the dynamic shared-memory limit only grows
    static std::mutex mu;
    if (smem > limit.load()) {
        std::lock_guard<std::mutex> lock(mu);
        if (smem > limit.load() &&
            cudaFuncSetAttribute(k_refresh_spec<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess)
            limit.store(smem);
    }
    k_refresh_spec<T><<<im.n_patches, kRedThreads, smem, st>>>(im, ch, part_lp, write_state);
    k_refresh_total<<<1, kRedThreads, 0, st>>>(part_ll, nblk, part_lp, im.n_patches, out_logpost, out_index);
    *launches += 3;
}
template void launch_refresh<float>(const Image&, const Chain&, double*, int, double*, const int*, int*, cudaStream_t,
                                    int64_t*);
template void launch_refresh<double>(const Image&, const Chain&, double*, int, double*, const int*, int*, cudaStream_t,
                                     int64_t*);

// ------------------------------------------------- photon-count draw -----
template <typename T>
__global__ void k_sample_phi(Image im, Chain ch, int t, int* err)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= im.H * im.W) return;
    const int a = idx / im.W, b = idx % im.W;
    const size_t k = (size_t)a * im.mu_pitch + b;
    const T mu = reinterpret_cast<const T*>(ch.mu)[k];
    const Dat4<T> dv = dat<T>(im)[idx];
    const uint4 x = philox4x32_10(make_uint4((uint32_t)idx, (uint32_t)t, (uint32_t)ch.chain, 1u), im.seed_lo,
                                  im.seed_hi);
    int status = 0;
    const int phi = sample_phi<T>(mu, dv.c, dv.is2, uniform23<T>(x.x), status);
    if (status) atomicOr(err, kErrNumeric);
    reinterpret_cast<T*>(ch.phi)[k] = (T)phi;
}

template <typename T>
void launch_sample_phi(const Image& im, const Chain& ch, int t, int* err, cudaStream_t st, int64_t* launches)
{
    const int n = im.H * im.W;
    k_sample_phi<T><<<(n + 255) / 256, 256, 0, st>>>(im, ch, t, err);
    ++*launches;
}
template void launch_sample_phi<float>(const Image&, const Chain&, int, int*, cudaStream_t, int64_t*);
template void launch_sample_phi<double>(const Image&, const Chain&, int, int*, cudaStream_t, int64_t*);

// ------------------------------------------------------------ reset -----
__global__ void k_reset(const Image* imgs, const Chain* chains, int n_slots)
{
    const Chain& ch = chains[blockIdx.x];
    const int np = imgs[ch.img].n_patches;
    for (int k = threadIdx.x; k < np; k += blockDim.x) ch.prog[(size_t)k * kProgStride] = 0;
    for (int k = threadIdx.x; k < n_slots * np; k += blockDim.x) ch.trace_part[k] = 0.0;
}

void launch_reset(const Image* d_imgs, const Chain* d_chains, int n_chains, int n_slots, cudaStream_t st,
                  int64_t* launches)
{
    k_reset<<<n_chains, 256, 0, st>>>(d_imgs, d_chains, n_slots);
    ++*launches;
}

// ------------------------------------------------------------ trace -----
// trace[t0 + s + 1] = trace[t0] + sum_{s' <= s} sum_p part[s'][p]: the double
// running sum of accepted dL + dP, per chain (one block per chain); t0 is the
// chain's sweep counter, which this kernel then advances by n.
__global__ void __launch_bounds__(kRedThreads) k_trace(const Image* imgs, const Chain* chains, int n)
{
    __shared__ double sh[kRedThreads];
    const Chain& ch = chains[blockIdx.x];
    const int np = imgs[ch.img].n_patches;
    const int t0 = *ch.tdev;
    double cum = ch.trace[t0];
    for (int s = 0; s < n; ++s) {
        double a = 0.0;
        for (int p = threadIdx.x; p < np; p += kRedThreads) a += ch.trace_part[(size_t)s * np + p];
        cum += block_sum(a, sh);
        if (threadIdx.x == 0) ch.trace[t0 + s + 1] = cum;
    }
    __syncthreads();
    if (threadIdx.x == 0) *ch.tdev = t0 + n;
}

void launch_trace(const Image* d_imgs, const Chain* d_chains, int n_chains, int n_sweeps, cudaStream_t st,
                  int64_t* launches)
{
    k_trace<<<n_chains, kRedThreads, 0, st>>>(d_imgs, d_chains, n_sweeps);
    ++*launches;
}

__global__ void k_set_counters(const Chain* chains, int n, int value)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) *chains[k].tdev = value;
}

void launch_set_counters(const Chain* d_chains, int n_chains, int value, cudaStream_t st, int64_t* launches)
{
    k_set_counters<<<(n_chains + 127) / 128, 128, 0, st>>>(d_chains, n_chains, value);
    ++*launches;
}

// --------------------------------------------------------- conversions --
template <typename T>
__global__ void k_to_double(const T* src, double* dst, int rows, int cols, int pitch)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)rows * cols) return;
    const int r = (int)(idx / cols), c = (int)(idx % cols);
    dst[idx] = (double)src[(size_t)r * pitch + c];
}

template <typename T>
void launch_convert(const void* src, double* dst, int64_t n, int rows, int cols, int src_pitch, cudaStream_t st,
                    int64_t* launches)
{
    (void)n;
    const int64_t tot = (int64_t)rows * cols;
    k_to_double<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(reinterpret_cast<const T*>(src), dst, rows, cols,
                                                                   src_pitch);
    ++*launches;
}
template void launch_convert<float>(const void*, double*, int64_t, int, int, int, cudaStream_t, int64_t*);
template void launch_convert<double>(const void*, double*, int64_t, int, int, int, cudaStream_t, int64_t*);

template <typename T>
__global__ void k_from_double(const double* src, T* dst, int64_t n)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) dst[idx] = (T)src[idx];
}

template <typename T>
void launch_set_rho(const double* src, void* dst, int64_t n, cudaStream_t st, int64_t* launches)
{
    k_from_double<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, reinterpret_cast<T*>(dst), n);
    ++*launches;
}
template void launch_set_rho<float>(const double*, void*, int64_t, cudaStream_t, int64_t*);
template void launch_set_rho<double>(const double*, void*, int64_t, cudaStream_t, int64_t*);

template <typename T>
__global__ void k_fill(T* dst, int64_t n, T value)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) dst[idx] = value;
}

template <typename T>
void launch_fill(void* dst, int64_t n, double value, cudaStream_t st, int64_t* launches)
{
    k_fill<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<T*>(dst), n, (T)value);
    ++*launches;
}
template void launch_fill<float>(void*, int64_t, double, cudaStream_t, int64_t*);
template void launch_fill<double>(void*, int64_t, double, cudaStream_t, int64_t*);

// posterior mean (variance, standard deviation, coefficient of variation)
// pooled over the chains of one problem
__global__ void k_mean(const double* sum, int n_chains, int64_t stride, int Wo, int crop_r, int oh, int ow,
                       double inv_n, double* out, const double* sq, int kind)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= oh * ow) return;
    const int y = idx / ow + crop_r, x = idx % ow + crop_r;
    const size_t m = (size_t)y * Wo + x;
    double s = 0.0, q = 0.0;
    for (int c = 0; c < n_chains; ++c) {
        s += sum[c * stride + m];
        if (kind) q += sq[c * stride + m];
    }
    const double mean = s * inv_n;
    if (kind == 0) {
        out[idx] = mean;
        return;
    }
    const double var = fmax(q * inv_n - mean * mean, 0.0);
    out[idx] = kind == 1 ? var : kind == 2 ? sqrt(var) : sqrt(var) / mean;
}

void launch_mean(const double* sum, int n_chains_img, int64_t chain_stride_elems, int Ho, int Wo, int crop_r,
                 int out_h, int out_w, double inv_n, double* out, const double* sq, int kind, cudaStream_t st,
                 int64_t* launches)
{
    (void)Ho;
    const int n = out_h * out_w;
    k_mean<<<(n + 255) / 256, 256, 0, st>>>(sum, n_chains_img, chain_stride_elems, Wo, crop_r, out_h, out_w, inv_n,
                                            out, sq, kind);
    ++*launches;
}

// ------------------------------------------------------------ quantiles --
// One block per output pixel: the pixel's kept values of every chain are
// loaded into shared memory, padded with +inf to a power of two, sorted by a
// bitonic network, and each requested quantile is read off the order
// statistics by linear interpolation at h = (n - 1) q.
template <typename T>
__global__ void __launch_bounds__(256) k_quantiles(const T* samples, int64_t chain_stride, int n_chains, int first,
                                                  int count, int64_t obj_pixels, int Wo, int crop_r, int out_w,
                                                  int64_t pix0, int npow2, const double* q, int nq, double* out,
                                                  int64_t npix)
{
    extern __shared__ double sv[];
    const int64_t i = blockIdx.x;
    const int64_t pix = pix0 + i;
    const int64_t y = pix / out_w + crop_r, x = pix % out_w + crop_r;
    const int64_t m = y * Wo + x;
    const int n = count * n_chains;
    for (int k = threadIdx.x; k < npow2; k += blockDim.x) {
        double v = INFINITY;
        if (k < n) {
            const int c = k / count, slot = first + (k - c * count);
            v = (double)samples[c * chain_stride + (int64_t)slot * obj_pixels + m];
        }
        sv[k] = v;
    }
    __syncthreads();
    for (int size = 2; size <= npow2; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int k = threadIdx.x; k < npow2 / 2; k += blockDim.x) {
                // element pair (a, b) of this stage, ascending where (a & size) == 0
                const int a = 2 * k - (k & (stride - 1)), b = a + stride;
                const bool up = (a & size) == 0;
                const double va = sv[a], vb = sv[b];
                if ((va > vb) == up) {
                    sv[a] = vb;
                    sv[b] = va;
                }
            }
            __syncthreads();
        }
    for (int k = threadIdx.x; k < nq; k += blockDim.x) {
        const double h = (double)(n - 1) * q[k];
        int lo = (int)floor(h);
        lo = lo < 0 ? 0 : lo > n - 1 ? n - 1 : lo;
        const int hi = lo + 1 < n ? lo + 1 : n - 1;
        out[(int64_t)k * npix + i] = sv[lo] + (h - (double)lo) * (sv[hi] - sv[lo]);
    }
}

template <typename T>
cudaError_t launch_quantiles(const void* samples, int64_t chain_stride, int n_chains, int first, int count,
                             int64_t obj_pixels, int Wo, int crop_r, int out_w, int64_t pix0, int64_t npix,
                             const double* q, int nq, double* out, cudaStream_t st, int64_t* launches)
{
    int npow2 = 2;
    while (npow2 < count * n_chains) npow2 <<= 1;
    const size_t smem = sizeof(double) * (size_t)npow2;
    cudaError_t e = cudaFuncSetAttribute((const void*)k_quantiles<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_quantiles<T><<<(unsigned)npix, 256, smem, st>>>(reinterpret_cast<const T*>(samples), chain_stride, n_chains,
                                                      first, count, obj_pixels, Wo, crop_r, out_w, pix0, npow2, q,
                                                      nq, out, npix);
    ++*launches;
    return cudaGetLastError();
}
template cudaError_t launch_quantiles<float>(const void*, int64_t, int, int, int, int64_t, int, int, int, int64_t,
                                             int64_t, const double*, int, double*, cudaStream_t, int64_t*);
template cudaError_t launch_quantiles<double>(const void*, int64_t, int, int, int, int64_t, int, int, int, int64_t,
                                              int64_t, const double*, int, double*, cudaStream_t, int64_t*);

}  // namespace bd
