// bd_sweep.cu -- persistent sub-lattice sweep kernel (the sampler's hot path).
//
// One thread block per tile of tpi x tpj prior patches of one chain; all
// blocks of all chains are co-resident (cooperative launch).  A sweep is the
// S*S classes (u, v) in raster order; the pixels of one class sit one per
// patch, S >= L apart, so their PSF windows are disjoint and each patch holds
// exactly one of them: given the rest of the object they are independent
// under Eq. 9 and are updated concurrently (Methods, "Parallelization
// Technique": the conditional of a point depends only on its neighbourhood).
// A tile starts class step s+1 only after the (up to 8) neighbouring tiles
// have finished step s, so every update sees exactly the state the
// sequential raster scan would give it; there is no grid-wide barrier.
//
// Each update is done by a team of im.team threads (fixed by the problem) with a fixed
// assignment of window pixels and spectrum entries and a fixed reduction
// tree, so results are bit-identical for every launch plan:
//   a2  Philox4x32-10 counter (m, t, chain, 0) -> z, u; rho' = rho e^{step z}
//   a4  dP = patch Dirichlet change (Eq. 7-8) with X'_k = X_k + delta w_k,
//       computed before waiting for the neighbours (it needs only the tile's
//       own spectrum)
//   a3  dL = sum over the L x L PSF window of the Eq. 6 change (dl_pixel),
//       the window's expected-image values fetched in one batch
//   a5  accept iff log u < dL + dP + step z; write rho, mu window, spectrum
//   a7  after the last class of a sweep: running sums of rho (double)
// The augmented sampler (AUG, BDECON_FLAG_AUGMENTED) starts every sweep with
// a photon-count step: each tile draws phi_n ~ p(phi | w_n, mu_n) for the
// camera pixels centred on its patches (after its neighbours finished the
// previous sweep), and a3 becomes the Poisson part of the completed
// likelihood (Eq. 5), sum_n phi_n log(1 + delta K / mu_n) - delta K, with no
// cumulant cache.
// In a resident plan the tile's per-pixel data constants (with the PSF halo),
// patch spectra and object values stay in shared memory for the launch; only
// mu, shared with the neighbouring tiles, is read from global memory (L2).
#include <type_traits>

#include <atomic>
#include <map>
#include <mutex>

#include "bd_device.cuh"

namespace bd {

// One entry of the patch prior change: X' = X + delta w, with
//   |X'|^2 - |X|^2 = delta (2 Re(X conj w) + delta)        (|w| = 1)
// accumulates  wa log(|X'|^2/|X|^2),  mult (|X'| - |X|),  mult |X|.
// The ratio form q = (|X'|^2 - |X|^2)/|X|^2 is free of cancellation while
// the coefficient does not shrink much (q > -1/2).  When it shrinks toward
// zero, q rounds to -1 (log1p = -inf, and with wa < 0 an infinite gain that
// the exact Eq. 7-8 change never has), so there the log is taken of the
// ratio |X'|^2/|X|^2 itself, with X' the value an accepted update stores.
// X' exactly 0 is rejected (the Dirichlet density is singular there).
template <typename T>
__device__ __forceinline__ void prior_term(T xr, T xi, T wr, T wi, T delta, T wa, T mult, T& accP, T& accS,
                                           T& accA, bool& bad)
{
    using P = Prec<T>;
    const T n2 = xr * xr + xi * xi;
    const T dd = delta * ((T)2 * (xr * wr + xi * wi) + delta);
    const T rn = fma(delta, wr, xr), in = fma(delta, wi, xi);
    const T n2n = rn * rn + in * in;
    if (!(n2n > (T)0)) bad = true;
    const T mo = P::sqrt(n2), mn = P::sqrt(n2n);
    const T i2 = P::rcp(n2);
    const T q = dd * i2;
    accP += wa * (q > (T)-0.5 ? P::log1p(q) : P::log(n2n * i2));
    accS += mult * (dd * P::rcp(mn + mo));
    accA += mult * mo;
}

// The target (Eq. 9) has a finite density at every state a chain can reach,
// so a proposal whose log acceptance ratio is not finite (and that is not
// impossible: mu' <= 0, a zero coefficient) is an arithmetic failure.  It is
// rejected, the numeric error bit raised, and the first such update recorded
// for the host: err[2] chain, err[3] pixel, err[8] sweep, dL and dP as
// doubles at err + 4.
__device__ __noinline__ void report_nonfinite(int* err, int chain, int m, int t, double dL, double dP)
{
    atomicOr(err, kErrRatio);
    if (atomicCAS(err + 1, 0, 1) == 0) {
        err[2] = chain;
        err[3] = m;
        err[8] = t;
        double* d = reinterpret_cast<double*>(err + 4);
        d[0] = dL;
        d[1] = dP;
    }
}

// x mod n for 0 <= x < 2^22 through a float reciprocal (exact after one correction)
__device__ __forceinline__ int small_mod(int x, int n, float inv_n)
{
    int r = x - n * __float2int_rz((float)x * inv_n);
    r += r < 0 ? n : 0;
    r -= r >= n ? n : 0;
    return r;
}

template <typename T>
__device__ __forceinline__ void twiddle(const T* tw, const Shape& sh, int kl, int u, int v, T& wr, T& wi)
{
    const int k = kl >> 16, l = kl & 0xffff;
    const T* eh = tw + 2 * (sh.twh_off + small_mod(k * u, sh.ph, sh.inv_ph));
    const T* ew = tw + 2 * (sh.tww_off + small_mod(l * v, sh.pw, sh.inv_pw));
    wr = eh[0] * ew[0] - eh[1] * ew[1];
    wi = eh[0] * ew[1] + eh[1] * ew[0];
}


// Window cell k (0 <= k < Lc^2) of object pixel (i, j): the camera pixel
// (aa, bb) it weighs on and the entry kw of the effective kernel Ke (Le x Le)
// with mu[aa][bb] = sum Ke[p][q] rho[f aa + Le-1-p][f bb + Le-1-q].  False
// when the cell is outside the frame (or, for f > 1, outside the kernel at
// this sub-cell phase).  f = 1 (FINE false): aa = i - 2R + k / L, kw = k.
template <bool FINE>
__device__ __forceinline__ bool win_cell(const Image& im, int i, int j, int k, int& aa, int& bb, int& kw)
{
    if (!FINE) {
        const int L = im.L, R = im.R;
        aa = i - 2 * R + k / L;
        bb = j - 2 * R + (k - (k / L) * L);
        kw = k;
        return k < L * L && (unsigned)aa < (unsigned)im.H && (unsigned)bb < (unsigned)im.W;
    }
    const int f = im.f, Le = im.Le, Lc = im.Lc;
    const int kr = k / Lc, kc = k - kr * Lc;
    aa = i / f - (Lc - 1) + kr;
    bb = j / f - (Lc - 1) + kc;
    const int p = f * aa + Le - 1 - i, q = f * bb + Le - 1 - j;
    kw = p * Le + q;
    return k < Lc * Lc && (unsigned)aa < (unsigned)im.H && (unsigned)bb < (unsigned)im.W && (unsigned)p < (unsigned)Le &&
           (unsigned)q < (unsigned)Le;
}

// a2: the proposal of one update from its Philox counter (m, t, chain, 0):
// z standard normal (Box-Muller), log u, the log-space move hz = s_m z (s_m
// the pixel's scale: its adapted one, else the problem's step) and
// rho' = rho exp(hz); hz is also the Hastings term of the decision.
template <typename T>
__device__ __forceinline__ void proposal(const Image& im, const Chain& ch, int m, int t, T r_old, T& hz, T& lu,
                                         T& r_new, T& delta)
{
    using P = Prec<T>;
    const uint4 x = philox4x32_10(make_uint4((uint32_t)m, (uint32_t)t, (uint32_t)ch.chain, 0u), im.seed_lo,
                                  im.seed_hi);
    const T z = P::gauss(uniform23<T>(x.x), uniform23<T>(x.y));
    const T sm = ch.steps != nullptr ? reinterpret_cast<const T*>(ch.steps)[m] : (T)im.step;
    hz = sm * z;
    lu = P::log(uniform23<T>(x.z));
    r_new = r_old * P::exp(hz);
    delta = r_new - r_old;
}

// Likelihood part of one update for one team thread: fetches the expected
// image (and, for float sweeps, the cached cumulants) of its window pixels
// in one batch, sums their Eq. 6 changes, and leaves the warp's partial sum
// and bad flag in out[0..1].  muv keeps the fetched expected image values.
// Fetch the first batch of a thread's window values (expected image and
// cached cumulants) so the loads are in flight while other work proceeds.
template <typename T, bool CUM, bool FINE, int NPX = kMaxPx>
__device__ __forceinline__ void window_fetch(const T* mu_g, const float4* cum_g, const float2* cum2_g,
                                             const Image& im, int i, int j, int lt, T (&muv)[NPX],
                                             float4 (&cq)[NPX], float2 (&cq2)[NPX], int k0)
{
    const int NT = im.team;
    // camera grid: the cell's row and column (k / L, k mod L) are advanced
    // from cell to cell (steps of NT) instead of divided out for each
    const int L = im.L;
    int kr = FINE ? 0 : k0 / L, kc = FINE ? 0 : k0 - kr * L;
    const int dr = FINE ? 0 : NT / L, dc = FINE ? 0 : NT - dr * L;
#pragma unroll
    for (int jj = 0; jj < NPX; ++jj) {
        const int k = k0 + jj * NT;
        int aa, bb, kw;
        bool in;
        if constexpr (FINE) {
            in = win_cell<FINE>(im, i, j, k, aa, bb, kw);
        } else {
            aa = i - 2 * im.R + kr;
            bb = j - 2 * im.R + kc;
            in = k < L * L && (unsigned)aa < (unsigned)im.H && (unsigned)bb < (unsigned)im.W;
            kc += dc;
            kr += dr;
            if (kc >= L) {
                kc -= L;
                ++kr;
            }
        }
        muv[jj] = in ? __ldcg(mu_g + (size_t)aa * im.mu_pitch + bb) : (T)-1;
        if (CUM) {
            cq[jj] = in ? __ldcg(cum_g + (size_t)aa * im.mu_pitch + bb) : make_float4(0, 0, 0, 0);
            cq2[jj] = in ? __ldcg(cum2_g + (size_t)aa * im.mu_pitch + bb) : make_float2(0, 0);
        }
    }
}

template <typename T, bool RES, bool CUM, bool FINE, int NPX = kMaxPx>
__device__ __forceinline__ void lik_partial(const T* mu_g, const float4* cum_g, const float2* cum2_g, const Dat4<T>* dat_s,
                                            const Dat4<T>* dat_g, const T* Ks, const Image& im, int i, int j,
                                            int a_lo, int b_lo, int rw, int lt, int NT, T delta, T (&muv)[NPX],
                                            T* out, int lane, float4 (&cq)[NPX], float2 (&cq2)[NPX],
                                            bool prefetched)
{
    const int W = im.W, LL = FINE ? im.Lc * im.Lc : im.L * im.L;
    T accL = 0;
    bool badL = false;
    for (int k0 = lt; k0 < LL; k0 += NT * NPX) {
        if (!(prefetched && k0 == lt)) window_fetch<T, CUM, FINE, NPX>(mu_g, cum_g, cum2_g, im, i, j, lt, muv, cq, cq2, k0);
#pragma unroll
        for (int jj = 0; jj < NPX; ++jj) {
            const int k = k0 + jj * NT;
            // on the camera grid the fetched window tells the cells apart (mu > 0
            // inside, -1 outside), so the geometry is needed only to read the
            // cell's data on the exact path; the finer lattice needs its PSF index
            int aa = 0, bb = 0, kw = k;
            const bool in = FINE ? win_cell<FINE>(im, i, j, k, aa, bb, kw) : muv[jj] != (T)-1;
            if (in) {
                const T xk = mul_rn(delta, Ks[kw]);
                if (CUM) {
                    const float d = (float)xk * Prec<float>::rcp((float)muv[jj]);
                    if (fabsf(d) <= kCumEval) {
                        accL += (T)cgf_delta((float)xk, log1p_cum(d), cq[jj], cq2[jj]);
                        continue;
                    }
                }
                if (!FINE) win_cell<FINE>(im, i, j, k, aa, bb, kw);
                const Dat4<T> dv = RES ? dat_s[(aa - a_lo) * rw + (bb - b_lo)] : dat_g[(size_t)aa * W + bb];
                if (CUM) {
                    int b = 0;
                    accL += (T)dl_pixel_call((float)muv[jj], (float)xk, (float)dv.c, (float)dv.is2, (float)dv.beta,
                                             &b);
                    badL = badL || b;
                } else {
                    accL += dl_pixel<T>(muv[jj], xk, dv.c, dv.is2, dv.beta, badL);
                }
            }
        }
    }
    accL = warp_sum(accL);
    const bool wb = __any_sync(0xffffffffu, badL);
    if (lane == 0) {
        out[0] = accL;
        out[1] = wb ? (T)1 : (T)0;
    }
}

// Likelihood part of one update for one team thread from the staged window
// (float marginal sampler, camera grid): the same cells in the same order
// with the same arithmetic as lik_partial, the expected image and the
// cumulants read from the shared-memory copy of the window (row stride BW,
// column offset dx of the window's first column within the copied box;
// cells outside the frame hold mu = 0).
template <bool RES>
__device__ __forceinline__ void lik_partial_staged(const float* wmu, const float4* wcum, const float2* wcum2, int BW,
                                                   int dx, const Dat4<float>* dat_s, const Dat4<float>* dat_g,
                                                   const float* Ks, const Image& im, int i, int j, int a_lo, int b_lo,
                                                   int rw, int lt, int NT, float delta, float* out, int lane)
{
    const int W = im.W, L = im.L, LL = L * L, R2 = 2 * im.R;
    float accL = 0.0f;
    bool badL = false;
    int kr = lt / L, kc = lt - (lt / L) * L;
    const int dr = NT / L, dc = NT - (NT / L) * L;
    for (int k = lt; k < LL; k += NT) {
        const int sidx = kr * BW + dx + kc;
        const float mu = wmu[sidx];
        if (mu > 0.0f) {
            const float xk = mul_rn(delta, Ks[k]);
            const float d = xk * Prec<float>::rcp(mu);
            if (fabsf(d) <= kCumEval) {
                accL += cgf_delta(xk, log1p_cum(d), wcum[sidx], wcum2[sidx]);
            } else {
                const int aa = i - R2 + kr, bb = j - R2 + kc;
                const Dat4<float> dv = RES ? dat_s[(aa - a_lo) * rw + (bb - b_lo)] : dat_g[(size_t)aa * W + bb];
                int b = 0;
                accL += dl_pixel_call(mu, xk, dv.c, dv.is2, dv.beta, &b);
                badL = badL || b;
            }
        }
        kc += dc;
        kr += dr;
        if (kc >= L) {
            kc -= L;
            ++kr;
        }
    }
    accL = warp_sum(accL);
    const bool wb = __any_sync(0xffffffffu, badL);
    if (lane == 0) {
        out[0] = accL;
        out[1] = wb ? 1.0f : 0.0f;
    }
}

// Augmented sampler: the window's expected image and photon counts.
template <typename T, bool FINE, int NPX = kMaxPx>
__device__ __forceinline__ void window_fetch_aug(const T* mu_g, const T* phi_g, const Image& im, int i, int j,
                                                 T (&muv)[NPX], T (&phv)[NPX], int k0)
{
    const int NT = im.team;
#pragma unroll
    for (int jj = 0; jj < NPX; ++jj) {
        const int k = k0 + jj * NT;
        int aa, bb, kw;
        const bool in = win_cell<FINE>(im, i, j, k, aa, bb, kw);
        muv[jj] = in ? __ldcg(mu_g + (size_t)aa * im.mu_pitch + bb) : (T)-1;
        phv[jj] = in ? __ldcg(phi_g + (size_t)aa * im.mu_pitch + bb) : (T)0;
    }
}

// Augmented sampler: the change of the Poisson part of the completed
// likelihood (Eq. 5) over the window at the current photon counts,
//   sum_n phi_n log(1 + delta K/mu_n) - delta K,
// a proposal making some mu'_n <= 0 being impossible.  Same thread
// assignment and reduction as lik_partial.
template <typename T, bool FINE, int NPX = kMaxPx>
__device__ __forceinline__ void lik_partial_aug(const T* mu_g, const T* phi_g, const T* Ks, const Image& im, int i,
                                                int j, int lt, int NT, T delta, T (&muv)[NPX], T (&phv)[NPX],
                                                T* out, int lane, bool prefetched)
{
    const int LL = FINE ? im.Lc * im.Lc : im.L * im.L;
    T accL = 0;
    bool badL = false;
    for (int k0 = lt; k0 < LL; k0 += NT * NPX) {
        if (!(prefetched && k0 == lt)) window_fetch_aug<T, FINE, NPX>(mu_g, phi_g, im, i, j, muv, phv, k0);
#pragma unroll
        for (int jj = 0; jj < NPX; ++jj) {
            const int k = k0 + jj * NT;
            int aa = 0, bb = 0, kw = k;
            const bool in = FINE ? win_cell<FINE>(im, i, j, k, aa, bb, kw) : muv[jj] != (T)-1;
            if (in) {
                const T xk = mul_rn(delta, Ks[kw]);
                const T d = xk / muv[jj];
                if (!(d > (T)-1)) {
                    badL = true;
                    continue;
                }
                T lg;
                if constexpr (std::is_same<T, float>::value) lg = log1p_cum(d);
                else lg = ::log1p(d);
                accL += phv[jj] * lg - xk;
            }
        }
    }
    accL = warp_sum(accL);
    const bool wb = __any_sync(0xffffffffu, badL);
    if (lane == 0) {
        out[0] = accL;
        out[1] = wb ? (T)1 : (T)0;
    }
}

// SOLO: a form compiled for plans in which every block updates one patch with
// one team (one round per step), without the multi-patch and multi-team paths
// STG: window staging (float marginal sampler on the camera grid, not the
// one-team form): each update's expected-image and cumulant window -- and, in
// streamed plans, its patch spectrum -- is copied into a shared-memory buffer
// of its team by the TMA engine, the next round's copy in flight while the
// current round computes (two buffers per team)
// LEAN: the float marginal camera-grid form (unstaged, not the one-team
// form) with half the window batch held in registers and a 64-register
// budget, for more resident warps per SM; the per-thread cell order, and so
// every result, is that of the other forms
template <typename T, bool RES, bool AUG, bool FINE, bool SOLO = false, int STG = 0, bool LEAN = false>
__global__ void __launch_bounds__(256, std::is_same<T, float>::value ? (LEAN ? 4 : 3) : 2) k_sweep(SweepArgs a)
{
    using P = Prec<T>;
    static_assert(!LEAN || (std::is_same<T, float>::value && !AUG && !FINE && !SOLO && STG == 0), "lean: float marginal camera grid");
    constexpr int NPX = LEAN ? kLeanPx : kMaxPx;
    // float sweeps of the marginal sampler use the cumulant cache; the
    // augmented sampler (AUG) scores windows from the photon counts instead
    constexpr bool CUM = std::is_same<T, float>::value && !AUG;
    static_assert(STG == 0 || (std::is_same<T, float>::value && !AUG && !FINE && !SOLO), "staging: float marginal camera grid");
    constexpr bool SANY = STG != 0;                          // staging
    constexpr bool SWIN = STG == 1;                          // the window is staged
    constexpr bool SSPEC = STG == 1 && !RES;                 // the patch spectrum is staged (streamed plans)
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_nbr[8];
    __shared__ int s_nn;
    __shared__ int s_abort;
    __shared__ int s_ci;
    __shared__ int s_stale;
    __shared__ int s_acc_any;
    __shared__ int s_pub;
    __shared__ int s_chg;   // the last published step changed data (thread 0 only)
    __shared__ int s_word;  // the last published progress word (thread 0 only)
    __shared__ double s_phid[AUG ? 8 : 1][8];   // photon-count step: [sub-team][warp] log-density changes
    __shared__ __align__(8) uint64_t s_bar;      // completion of the tile's bulk copies (resident plans)

    const int tid = threadIdx.x;
    if (tid == 0) {
        int lo = 0, hi = a.n_chains - 1;
        while (lo < hi) {   // last chain with cta_base <= blockIdx.x
            const int mid = (lo + hi + 1) >> 1;
            if (a.chains[mid].cta_base <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
        }
        s_ci = lo;
    }
    __syncthreads();
    // the chain and problem descriptors are copied to shared memory: the step
    // loop reads them at every step, and after each neighbour wait's acquire
    // fence they would otherwise be fetched from L2 again
    __shared__ __align__(16) uint32_t s_chd[sizeof(Chain) / 4];
    __shared__ __align__(16) uint32_t s_imd[sizeof(Image) / 4];
    static_assert(sizeof(Chain) % 4 == 0 && sizeof(Image) % 4 == 0, "descriptor copies are whole words");
    {
        const uint32_t* gc = reinterpret_cast<const uint32_t*>(&a.chains[s_ci]);
        const uint32_t* gi = reinterpret_cast<const uint32_t*>(&a.imgs[a.chains[s_ci].img]);
        for (int k = tid; k < (int)(sizeof(Chain) / 4); k += blockDim.x) s_chd[k] = gc[k];
        for (int k = tid; k < (int)(sizeof(Image) / 4); k += blockDim.x) s_imd[k] = gi[k];
    }
    __syncthreads();
    const Chain& ch = *reinterpret_cast<const Chain*>(s_chd);
    const Image& im = *reinterpret_cast<const Image*>(s_imd);
    const int t0 = *ch.tdev;          // sweeps completed before this launch (advanced after it by k_trace)
    const int tl = (int)blockIdx.x - ch.cta_base;
    const int ti = tl / ch.ntj, tj = tl - (tl / ch.ntj) * ch.ntj;
    const int S = im.S, L = im.L, R = im.R, H = im.H, W = im.W, S2 = S * S;
    // lattice f times finer than the camera (FINE; f = 1 otherwise): LL window cells per update
    const int f = FINE ? im.f : 1, Le = FINE ? im.Le : L, Lc = FINE ? im.Lc : L, LL = Lc * Lc;
    const int pi0 = SOLO ? ti : ti * ch.tpi, pj0 = SOLO ? tj : tj * ch.tpj;
    const int pi1 = SOLO ? pi0 + 1 : min(pi0 + ch.tpi, im.npi), pj1 = SOLO ? pj0 + 1 : min(pj0 + ch.tpj, im.npj);
    const int tw_ = SOLO ? 1 : pj1 - pj0, npt = SOLO ? 1 : (pi1 - pi0) * tw_;
    // camera region seen by the tile's windows
    const int i0 = pi0 * S, j0 = pj0 * S, i1 = min(pi1 * S, im.Ho), j1 = min(pj1 * S, im.Wo);
    const int a_lo = !FINE ? max(0, i0 - 2 * R) : max(0, i0 / f - (Lc - 1));
    const int a_hi = !FINE ? min(H, i1) : min(H, (i1 - 1) / f + 1);
    const int b_lo = !FINE ? max(0, j0 - 2 * R) : max(0, j0 / f - (Lc - 1));
    const int b_hi = !FINE ? min(W, j1) : min(W, (j1 - 1) / f + 1);
    const int rw = b_hi - b_lo;

    const SmemPlan sp = smem_plan(L, f, S, im.n_tw, im.n_ent, im.max_nhalf, ch.tpi, ch.tpj, RES ? 1 : 0, sizeof(T),
                                  max(1, (int)blockDim.x / im.team), STG, LEAN);
    const StagePlan stp = stage_plan(L, im.max_nhalf, STG, RES ? 1 : 0);
    const int BW = stage_w(L);
    uint64_t* stg_bar = reinterpret_cast<uint64_t*>(smem + sp.stage_bar);   // [team][buffer]
    T* red = reinterpret_cast<T*>(smem + sp.red);          // [2][8 sub-teams][8 warps][4]
    T* Ks = reinterpret_cast<T*>(smem + sp.K);
    T* tws = reinterpret_cast<T*>(smem + sp.tw);
    int* ekl = reinterpret_cast<int*>(smem + sp.ekl);
    T* ewa = reinterpret_cast<T*>(smem + sp.ewa);
    T* em = reinterpret_cast<T*>(smem + sp.em);
    T* ring = reinterpret_cast<T*>(smem + sp.prop);         // [team][kPropRing][4]
    T* spec_s = reinterpret_cast<T*>(smem + sp.spec);       // [npt][max_nhalf] complex
    T* rho_s = reinterpret_cast<T*>(smem + sp.rho);         // [npt][S*S]
    Dat4<T>* dat_s = reinterpret_cast<Dat4<T>*>(smem + sp.dat);

    T* rho_g = reinterpret_cast<T*>(ch.rho);
    T* mu_g = reinterpret_cast<T*>(ch.mu);
    T* phi_g = reinterpret_cast<T*>(ch.phi);
    T* spec_g = reinterpret_cast<T*>(ch.spec);
    float4* cum_g = ch.cum;
    float2* cum2_g = ch.cum2;
    const Dat4<T>* dat_g = dat<T>(im);

    // ---- prologue: neighbours, tables, resident tile state
    if (tid == 0) {
        int nn = 0;
        for (int di = -1; di <= 1; ++di)
            for (int dj = -1; dj <= 1; ++dj) {
                const int ni = ti + di, nj = tj + dj;
                if ((di || dj) && ni >= 0 && ni < ch.nti && nj >= 0 && nj < ch.ntj) s_nbr[nn++] = ni * ch.ntj + nj;
            }
        s_nn = nn;
        s_abort = 0;
        s_stale = 0;
        s_acc_any = 0;
        s_pub = 0;
        s_chg = 0;
        s_word = 0;
        if (RES) mbar_init(&s_bar, 1);
        if (SANY)
            for (int k = 0; k < 2 * max(1, (int)blockDim.x / im.team); ++k) mbar_init(&stg_bar[k], 1);
    }
    // Resident plans: the tile's per-pixel constants -- camera rows a_lo..a_hi-1,
    // columns b_lo..b_hi-1, i.e. the tile's windows with the PSF halo -- are
    // staged in shared memory by bulk copies of the TMA engine, one per row (rw
    // records of 16 or 32 bytes, 16-byte-aligned at both ends), issued by the
    // first warp and overlapped with the table loads below
    const int n_rows = RES ? a_hi - a_lo : 0;
    const bool staged = RES && n_rows > 0 && rw > 0;
    if (RES) {
        __syncthreads();   // barrier initialised
        if (staged && tid < 32) {
            const uint32_t row_bytes = (uint32_t)rw * (uint32_t)sizeof(Dat4<T>);
            if (tid == 0) mbar_arrive_expect_tx(&s_bar, (uint32_t)n_rows * row_bytes);
            __syncwarp();
            for (int r = tid; r < n_rows; r += 32)
                bulk_g2s(dat_s + (size_t)r * rw, dat_g + (size_t)(a_lo + r) * W + b_lo, row_bytes, &s_bar);
        }
    }
    for (int k = tid; k < Le * Le; k += blockDim.x) Ks[k] = kern<T>(im)[k];
    for (int k = tid; k < 2 * im.n_tw; k += blockDim.x) tws[k] = twid<T>(im)[k];
    for (int k = tid; k < im.n_ent; k += blockDim.x) {
        ekl[k] = im.ent_kl[k];
        ewa[k] = ent_wa<T>(im)[k];
        em[k] = ent_m<T>(im)[k];
    }
    if (RES) {
        for (int q = 0; q < npt; ++q) {
            const int pi = pi0 + q / tw_, pj = pj0 + (q - (q / tw_) * tw_);
            const Shape& sh = im.shape[shape_index(im, pi, pj)];
            const T* src = spec_g + 2 * im.patch_off[pi * im.npj + pj];
            for (int e = tid; e < 2 * sh.nhalf; e += blockDim.x) spec_s[(size_t)q * 2 * im.max_nhalf + e] = src[e];
            for (int e = tid; e < sh.ph * sh.pw; e += blockDim.x) {
                const int uu = e / sh.pw, vv = e - (e / sh.pw) * sh.pw;
                rho_s[(size_t)q * S2 + uu * S + vv] = rho_g[(size_t)(pi * S + uu) * im.Wo + pj * S + vv];
            }
        }
    }
    if (staged && !mbar_wait(&s_bar, 0, a.wait_ns)) {
        atomicOr(a.err, kErrTimeout);
        s_abort = 1;
    }
    __syncthreads();
    if (s_abort) {
        // the copies were not seen to land: give them one more bounded wait
        // before the block's shared memory is released
        if (staged) (void)mbar_wait(&s_bar, 0, a.wait_ns);
        return;
    }

    const int NT = im.team;
    const int n_sub = SOLO ? 1 : max(1, (int)blockDim.x / NT);
    const int g = SOLO ? 0 : tid / NT, lt = SOLO ? tid : tid - (tid / NT) * NT;
    const bool in_team = SOLO || g < n_sub;
    const int twarp = lt >> 5, lane = tid & 31, nwt = NT >> 5;
    const int rounds = SOLO ? 1 : (npt + n_sub - 1) / n_sub;
    T* red1 = red + (size_t)(g * 8) * 4;                   // prior partials of this sub-team
    T* red2 = red + 8 * 8 * 4 + (size_t)(g * 8) * 4;       // likelihood partials
    // a sweep is S2 class steps, preceded in the augmented sampler by a
    // photon-count step (so SS = S2 + 1 steps); cs counts class steps only
    const int SS = AUG ? S2 + 1 : S2;
    const int nsw = ch.n_sweeps > 0 ? ch.n_sweeps : a.n_sweeps;
    const int nsteps = nsw * SS, ncs = nsw * S2;
    int n_acc = 0;
    // a warp of each team draws the team's proposals ahead of time, between
    // the step barriers (while the polling warp waits for the neighbours), into
    // the ring.  Updates are numbered by round ordinal e = class step x rounds
    // + round; the draw of update e uses the pixel's rho and scale, which
    // change only at the pixel's own previous update, e - S^2 rounds, so a draw
    // made fewer than S^2 rounds ahead is exact.  With more than kPropRing
    // rounds per sweep the warp's lanes draw the next kPropRing updates
    // together (wide), else the whole warp draws the next one.  Not when a
    // sweep is a single round (S = 1 and one round), where the next update
    // revisits the pixel.
    // Blocks of two update teams with several rounds per class step (tb):
    // after the first round of a step the teams share nothing until the step
    // ends -- their patches, windows, partial sums, proposal rings and staging
    // buffers are their own -- so in those rounds each team synchronises alone
    // (tsync, a named barrier per team; threads outside both teams take no
    // part), a team does not wait for the other's slower round, and the block
    // meets again at the step's end.  Other plans use block barriers throughout.
    const bool tb = !SOLO && n_sub == 2 && rounds > 1;
    auto tsync = [&]() {
        if (in_team) team_bar2(g, NT);
    };
    const int SR = S2 * rounds;   // rounds per sweep
    const bool ahead = SR > 1;
    // In those team-barrier rounds of unstaged forms the second team barrier
    // (after the decision) is dropped (nob2): the round's partial sums alternate
    // between two buffers by round parity, so the next round's writes cannot
    // meet this round's reads (a team reaches the next round's first barrier
    // only when all its threads finished this round's decision), and proposals
    // are drawn two rounds ahead, so a draw is published by the first barrier
    // of the round before its own.  Needs more than two rounds per sweep (the
    // draw two ahead must not be the current pixel's next update).
    // (the lean form only: in the other forms the extra code costs more than
    // the barrier -- measured)
    const bool nob2 = LEAN && tb && SR > 2;
    const int RB = 2 * 8 * 8 * 4;   // one set of partial sums
    const int pwarp = nwt > 1 ? 1 : 0;   // the drawing warp: not the one that polls the flags
    // one update per block and step (rounds == 1, n_sub == 1): a rejected
    // update scored on the neighbours' final state leaves nothing to write or
    // reread, so thread 0 publishes the step as soon as its wait ends
    // (s_pub: already published; thread 0 only)
    // wide: with more than kPropRing rounds per sweep the warp's lanes draw
    // several updates together, one each: the next kPropRing at every
    // kPropRing-th round, or, two ahead (nob2), the next 16 at every 16th
    const bool wide = SR > kPropRing;
    auto draw_ahead = [&](int e0) {
        const int e = e0 + (wide ? lane : 0);            // round ordinal of the draw
        const int cs_e = e / rounds, r_e = e - cs_e * rounds;
        const int q = r_e * n_sub + g;                   // this team's patch in that round
        const int sw = cs_e / S2, cl = cs_e - sw * S2;
        const int u1 = cl / S, v1 = cl - (cl / S) * S;
        if (cs_e < ncs && q < npt) {
            const int pi_ = pi0 + q / tw_, pj_ = pj0 + (q - (q / tw_) * tw_);
            const Shape& sh1 = im.shape[shape_index(im, pi_, pj_)];
            if (u1 < sh1.ph && v1 < sh1.pw) {
                const int m1 = (pi_ * S + u1) * im.Wo + pj_ * S + v1;
                T z1, lu1, rn1, dl1;
                proposal<T>(im, ch, m1, t0 + 1 + sw, RES ? rho_s[(size_t)q * S2 + u1 * S + v1] : rho_g[m1], z1,
                            lu1, rn1, dl1);
                if (wide || lane == 0) {
                    T* pe = ring + ((size_t)g * kPropRing + (e & (kPropRing - 1))) * 4;
                    pe[0] = z1; pe[1] = lu1; pe[2] = rn1; pe[3] = dl1;
                }
            }
        }
    };
    // (lean form: the first n lanes only, when wide)
    auto draw_ahead_n = [&](int e0, int n) {
        if (wide && lane >= n) return;
        const int e = e0 + (wide ? lane : 0);            // round ordinal of the draw
        const int cs_e = e / rounds, r_e = e - cs_e * rounds;
        const int q = r_e * n_sub + g;                   // this team's patch in that round
        const int sw = cs_e / S2, cl = cs_e - sw * S2;
        const int u1 = cl / S, v1 = cl - (cl / S) * S;
        if (cs_e < ncs && q < npt) {
            const int pi_ = pi0 + q / tw_, pj_ = pj0 + (q - (q / tw_) * tw_);
            const Shape& sh1 = im.shape[shape_index(im, pi_, pj_)];
            if (u1 < sh1.ph && v1 < sh1.pw) {
                const int m1 = (pi_ * S + u1) * im.Wo + pj_ * S + v1;
                T z1, lu1, rn1, dl1;
                proposal<T>(im, ch, m1, t0 + 1 + sw, RES ? rho_s[(size_t)q * S2 + u1 * S + v1] : rho_g[m1], z1,
                            lu1, rn1, dl1);
                if (wide || lane == 0) {
                    T* pe = ring + ((size_t)g * kPropRing + (e & (kPropRing - 1))) * 4;
                    pe[0] = z1; pe[1] = lu1; pe[2] = rn1; pe[3] = dl1;
                }
            }
        }
    };
    // Window staging (STG).  Round ordinal e of this team uses buffer e & 1;
    // the copy set of round e + 1 is issued while round e computes, except
    // that the first round of a class step is issued after the previous step's
    // writes (its windows overlap them) and, like the register path's
    // speculative fetch, is re-copied when the neighbour wait finds it stale.
    // Issue and wait conditions are the same predicate, so each barrier's
    // phases stay in step; stg_par holds the parity to wait for per buffer and
    // stg_pend the buffers with a copy in flight (both uniform in a team).
    uint32_t stg_par = 0, stg_pend = 0;
    auto stg_buf = [&](int b) { return smem + sp.stage + ((size_t)g * 2 + b) * stp.per_buf; };
    auto stage_issue = [&](int e) -> bool {
        if (!SANY || !in_team) return false;
        const int cs_e = e / rounds, r_e = e - cs_e * rounds;
        const int q = r_e * n_sub + g;
        if (cs_e >= ncs || q >= npt) return false;
        const int cl = cs_e - (cs_e / S2) * S2;
        const int u1 = cl / S, v1 = cl - (cl / S) * S;
        const int pi_ = pi0 + q / tw_, pj_ = pj0 + (q - (q / tw_) * tw_);
        const Shape& sh1 = im.shape[shape_index(im, pi_, pj_)];
        if (u1 >= sh1.ph || v1 >= sh1.pw) return false;
        const int b = e & 1;
        if (lt == 0) {
            unsigned char* buf = stg_buf(b);
            uint64_t* bar = &stg_bar[g * 2 + b];
            const int x0 = (pj_ * S + v1 - 2 * R) & ~3, y0 = pi_ * S + u1 - 2 * R;
            const uint32_t spec_bytes = SSPEC ? (uint32_t)((sh1.nhalf + 1) & ~1) * 8u : 0u;
            const char* tm = reinterpret_cast<const char*>(ch.tmap);
            fence_proxy_async_global();
            mbar_arrive_expect_tx(bar, (SWIN ? stp.tx_win : 0u) + spec_bytes);
            if (SWIN) {
                tma_load_2d(buf + stp.mu, tm, x0, y0, bar);
                tma_load_2d(buf + stp.cum, tm + 128, 4 * x0, y0, bar);
                tma_load_2d(buf + stp.cum2, tm + 256, 2 * x0, y0, bar);
            }
            if (SSPEC) bulk_g2s(buf + stp.spec, spec_g + 2 * im.patch_off[pi_ * im.npj + pj_], spec_bytes, bar);
        }
        stg_pend |= 1u << b;
        return true;
    };
    auto stage_wait = [&](int b) {
        const bool ok = mbar_wait(&stg_bar[g * 2 + b], (stg_par >> b) & 1u, a.wait_ns);
        stg_par ^= 1u << b;
        stg_pend &= ~(1u << b);
        if (!ok) {
            atomicOr(a.err, kErrTimeout);
            s_abort = 1;
        }
    };
    // before the block returns: copies still in flight must land first (bounded)
    auto stage_drain = [&]() {
        for (int b = 0; b < 2; ++b)
            if ((stg_pend >> b) & 1u) stage_wait(b);
    };
    if (SANY) stage_issue(0);
    if (ahead && in_team && twarp == pwarp) {
        if constexpr (LEAN) {
            if (wide) {
                draw_ahead_n(0, nob2 ? 18 : kPropRing);
            } else {
                draw_ahead_n(0, 1);
                if (nob2) draw_ahead_n(1, 1);
            }
        } else {
            draw_ahead(0);
        }
    }
    __syncthreads();

    for (int s = 0; s < nsteps; ++s) {
        const int slot = s / SS, cc = s - slot * SS;
        const int t = t0 + 1 + slot;
        if constexpr (AUG) {
            if (cc == 0) {
                // a0 (augmented sampler): after the neighbours finished the previous
                // sweep, draw the photon counts of the camera pixels centred on the
                // tile's patches from p(phi | w, mu) (Philox counter (n, t, chain, 1));
                // the change of the log joint density goes to the patch's trace part
                if (s > 0 && tid < 32) {
                    int word;
                    const bool ok = warp_wait_flags(ch.prog, s_nbr, s_nn, s, a.err, a.wait_ns, word);
                    fence_acq_rel_gpu();
                    if (lane == 0 && !ok) s_abort = 1;
                }
                __syncthreads();
                if (s_abort) return;
                for (int r = 0; r < rounds; ++r) {
                    const int q = r * n_sub + g;
                    double dj = 0.0;
                    int pi = 0, pj = 0;
                    if (in_team && q < npt) {
                        pi = pi0 + q / tw_;
                        pj = pj0 + (q - (q / tw_) * tw_);
                        const Shape& shp = im.shape[shape_index(im, pi, pj)];
                        int bad = 0;
                        for (int e = lt; e < shp.ph * shp.pw; e += NT) {
                            // the camera pixel anchored at this object pixel: object row
                            // f a + R (f = 1: every object pixel anchors one)
                            const int uu = e / shp.pw, vv = e - (e / shp.pw) * shp.pw;
                            const int ir = pi * S + uu - R, jr = pj * S + vv - R;
                            if (ir < 0 || jr < 0 || ir % f != 0 || jr % f != 0) continue;
                            const int aa = ir / f, bb = jr / f;
                            if (aa >= H || bb >= W) continue;
                            const size_t idx = (size_t)aa * im.mu_pitch + bb;
                            const T mu = __ldcg(mu_g + idx);
                            const Dat4<T> dv = RES ? dat_s[(aa - a_lo) * rw + (bb - b_lo)] : dat_g[(size_t)aa * W + bb];
                            const uint4 x = philox4x32_10(
                                make_uint4((uint32_t)(aa * W + bb), (uint32_t)t, (uint32_t)ch.chain, 1u), im.seed_lo,
                                im.seed_hi);
                            const int pn = sample_phi<T>(mu, dv.c, dv.is2, uniform23<T>(x.x), bad);
                            const int po = (int)phi_g[idx];
                            const double lmu = ::log((double)mu);
                            dj += phi_logterm(pn, lmu, (double)dv.c, (double)dv.is2) -
                                  phi_logterm(po, lmu, (double)dv.c, (double)dv.is2);
                            phi_g[idx] = (T)pn;
                        }
                        if (bad) atomicOr(a.err, kErrNumeric);
                        dj = warp_sum(dj);
                        if (lane == 0) s_phid[g][twarp] = dj;
                    }
                    __syncthreads();
                    if (in_team && q < npt && lt == 0) {
                        double tot = 0.0;
                        for (int w = 0; w < nwt; ++w) tot += s_phid[g][w];
                        ch.trace_part[(size_t)slot * im.n_patches + pi * im.npj + pj] += tot;
                    }
                    __syncthreads();
                }
                if (tid == 0 && (int)blockIdx.x != a.silent_block) {
                    // the neighbours' next windows read these counts: mark the step
                    // changed (their speculative scores are redone) and release
                    const int w = prog_word(s + 1, true, s_chg != 0);
                    red_add_release(ch.prog + (size_t)tl * kProgStride, w - s_word);
                    s_word = w;
                    s_chg = 1;
                }
                continue;
            }
        }
        const int c = AUG ? cc - 1 : cc;
        const int cs = slot * S2 + c;            // class-step ordinal
        const int u = c / S, v = c - (c / S) * S;
        // one-team form: the polling warp reads the neighbours' progress words
        // at the start of the step, so that the load overlaps the step's own
        // work; the wait polls again only if a neighbour had not yet published
        // the previous step (words only grow, and carry the change marks)
        int pre = 0;
        if constexpr (SOLO) {
            if (s > 0 && tid < 32 && lane < s_nn) pre = ld_relaxed(ch.prog + (size_t)s_nbr[lane] * kProgStride);
        }
        for (int r = 0; r < rounds; ++r) {
            const int q = r * n_sub + g;
            bool active = in_team && q < npt;
            int pi = 0, pj = 0, sidx = 0;
            if (active) {
                pi = pi0 + q / tw_;
                pj = pj0 + (q - (q / tw_) * tw_);
                sidx = shape_index(im, pi, pj);
                active = u < im.shape[sidx].ph && v < im.shape[sidx].pw;
            }
            const Shape& sh = im.shape[sidx];
            const int i = pi * S + u, j = pj * S + v;
            const int m = i * im.Wo + j;
            T z = 0, lu = 0, r_old = 0, r_new = 0, delta = 0;
            bool badP = false;
            T* spec_p = RES ? spec_s + (size_t)q * 2 * im.max_nhalf : spec_g + 2 * im.patch_off[pi * im.npj + pj];
            T muv[NPX];
            float4 cq[AUG ? 1 : NPX];
            float2 cq2[AUG ? 1 : NPX];
            T phv[AUG ? NPX : 1];
            // staged window of this round (STG): buffer e & 1 of the team
            const int e_cur = cs * rounds + r, sb = e_cur & 1;
            // this round's partial sums (alternating sets in nob2 rounds)
            T* pr1 = red1;
            T* pr2 = red2;
            if constexpr (LEAN) {
                if (nob2) {
                    pr1 += (size_t)(e_cur & 1) * RB;
                    pr2 += (size_t)(e_cur & 1) * RB;
                }
            }
            const float* wmu = reinterpret_cast<const float*>(stg_buf(sb) + stp.mu);
            const float4* wcum = reinterpret_cast<const float4*>(stg_buf(sb) + stp.cum);
            const float2* wcum2 = reinterpret_cast<const float2*>(stg_buf(sb) + stp.cum2);
            const int wdx = (j - 2 * R) - ((j - 2 * R) & ~3);
            // spectrum read here (the staged copy in streamed STG plans); writes go to spec_p
            const T* spec_rd = SSPEC ? reinterpret_cast<const T*>(stg_buf(sb) + stp.spec) : spec_p;
            if constexpr (SANY) {
                if (active) stage_wait(sb);
                // the next round of this step: its window is disjoint from this one
                // (same class, another patch), so its copy overlaps this round's work
                if (r >= 1 && r + 1 < rounds) stage_issue(e_cur + 1);
            }
            // the window's first batch is fetched before the prior work so its
            // latency overlaps the arithmetic below
            if (active && !SWIN) {
                if constexpr (AUG) window_fetch_aug<T, FINE, NPX>(mu_g, phi_g, im, i, j, muv, phv, lt);
                else window_fetch<T, CUM, FINE, NPX>(mu_g, cum_g, cum2_g, im, i, j, lt, muv, cq, cq2, lt);
            }
            // a2 + a4: proposal and prior change (own tile state only)
            if (active) {
                if (ahead) {
                    const int e = cs * rounds + r;
                    const T* pe = ring + ((size_t)g * kPropRing + (e & (kPropRing - 1))) * 4;
                    z = pe[0];
                    lu = pe[1];
                    r_new = pe[2];
                    delta = pe[3];
                } else {
                    r_old = RES ? rho_s[(size_t)q * S2 + u * S + v] : rho_g[m];
                    proposal<T>(im, ch, m, t, r_old, z, lu, r_new, delta);
                }
                T accP = 0, accS = 0, accA = 0;
                for (int e = lt; e < sh.nhalf; e += NT) {
                    T wr, wi;
                    const int ent = sh.ent_off + e;
                    twiddle(tws, sh, ekl[ent], u, v, wr, wi);
                    prior_term<T>(spec_rd[2 * e], spec_rd[2 * e + 1], wr, wi, delta, ewa[ent], em[ent], accP, accS,
                                  accA, badP);
                }
                accP = warp_sum(accP);
                accS = warp_sum(accS);
                accA = warp_sum(accA);
                const bool wb = __any_sync(0xffffffffu, badP);
                if (lane == 0) {
                    pr1[twarp * 4 + 0] = accP;
                    pr1[twarp * 4 + 1] = accS;
                    pr1[twarp * 4 + 2] = accA;
                    pr1[twarp * 4 + 3] = wb ? (T)1 : (T)0;
                }
            }
            // a3: likelihood change over the PSF window.  For the first round of
            // a step this runs before the neighbour wait, on the expected image
            // as it is now; it is redone below only if a neighbouring tile
            // accepted an update since this block last waited for it.
            if (active) {
                if constexpr (AUG)
                    lik_partial_aug<T, FINE, NPX>(mu_g, phi_g, Ks, im, i, j, lt, NT, delta, muv, phv, pr2 + twarp * 4, lane,
                                             true);
                else if constexpr (SWIN)
                    lik_partial_staged<RES>(wmu, wcum, wcum2, BW, wdx, dat_s, dat_g, Ks, im, i, j, a_lo, b_lo, rw, lt,
                                            NT, delta, pr2 + twarp * 4, lane);
                else
                    lik_partial<T, RES, CUM, FINE, NPX>(mu_g, cum_g, cum2_g, dat_s, dat_g, Ks, im, i, j, a_lo, b_lo, rw, lt, NT,
                                             delta, muv, pr2 + twarp * 4, lane, cq, cq2, true);
            }
            // a5: Metropolis-Hastings decision with the Hastings term of the log-space
            // walk, taken from the round's partial sums as soon as every warp of the
            // team has written them -- before the neighbour wait, so that a rejected
            // update (the common case) leaves only the wait and the publish after it.
            // In the first round the whole block meets: every thread has then read
            // the previous step's stale and abort flags, which the polling warp
            // is about to overwrite
            if (r == 0 || !tb) __syncthreads();
            else tsync();
            T dL = 0, dP = 0;
            bool accept = false, nonfin = false;
            auto decide = [&]() {
                T sP = 0, sS = 0, sA = 0;
                bool bad = false;
                dL = 0;
                for (int w = 0; w < nwt; ++w) {
                    sP += pr1[w * 4 + 0];
                    sS += pr1[w * 4 + 1];
                    sA += pr1[w * 4 + 2];
                    bad = bad || pr1[w * 4 + 3] != (T)0;
                    dL += pr2[w * 4 + 0];
                    bad = bad || pr2[w * 4 + 1] != (T)0;
                }
                dP = sP + (T)(sh.K - 1) * P::log1p(sS / sA);
                const T tot = dL + dP;
                nonfin = !bad && !(fabs(tot) <= (T)P::kMaxFinite);
                accept = !bad && !nonfin && (lu < tot + z);   // z holds s_m z
            };
            if (active) decide();
            // the next step's draw, after the step barrier so that the other warps
            // need not wait for it there; it overlaps the neighbour wait below
            if (ahead && in_team && twarp == pwarp) {
                const int e = cs * rounds + r;
                if constexpr (LEAN) {
                    if (!wide) draw_ahead_n(e + (nob2 ? 2 : 1), 1);
                    else if (nob2) { if ((e & 15) == 0 && e > 0) draw_ahead_n(e + 2, 16); }
                    else if ((e & (kPropRing - 1)) == kPropRing - 1) draw_ahead_n(e + 1, kPropRing);
                } else {
                    if (!wide || (e & (kPropRing - 1)) == kPropRing - 1) draw_ahead(e + 1);
                }
            }
            if (r == 0 && s > 0 && tid < 32) {
                // stale: a neighbour changed data this window reads at its step s-1
                // (or at step s, whose windows are disjoint from this one: a
                // harmless recompute), read from the word the wait ended on
                int word;
                const bool ok = warp_wait_flags(ch.prog, s_nbr, s_nn, s, a.err, a.wait_ns, word, pre);
                bool stale = false;
                if (ok && lane < s_nn) stale = (word & ((word >> 2) > s ? 3 : 1)) != 0;
                stale = __any_sync(0xffffffffu, stale);
                // acquire only when a neighbour changed data since this block's
                // last acquire: otherwise nothing read after this wait was
                // written by a neighbour since then (this step's reads came
                // before the wait, and a neighbour's change at step s is marked
                // in the words of the next wait)
                if (stale) fence_acq_rel_gpu();
                if (lane == 0) {
                    if (!ok) s_abort = 1;
                    s_stale = stale ? 1 : 0;
                    if (ok && !stale && !accept && rounds == 1 && n_sub == 1 && (int)blockIdx.x != a.silent_block) {
                        const int w = prog_word(s + 1, false, s_chg != 0);
                        red_add_relaxed(ch.prog + (size_t)tl * kProgStride, w - s_word);
                        s_word = w;
                        s_chg = 0;
                        s_pub = 1;
                    }
                }
            }
            // (the partial sums are not read after this barrier, so the next round
            // may overwrite them; writes of an accepted update need one more)
            // (one-team form: every thread took the same decision, so a plain
            // barrier does; team barriers: a team's decision is uniform in it)
            const bool blk = r == 0 || !tb;
            int any_accept;
            if constexpr (SOLO) {
                __syncthreads();
                any_accept = active && accept ? 1 : 0;
            } else if (blk) {
                any_accept = __syncthreads_or(active && accept ? 1 : 0);
            } else {
                if constexpr (LEAN) {
                    if (!nob2) tsync();
                } else {
                    tsync();
                }
                any_accept = active && accept ? 1 : 0;
            }
            if (blk && s_abort) {
                stage_drain();
                return;
            }
            const bool stale = r == 0 && s > 0 && s_stale;
            if (stale) {
                if (active) {
                    if constexpr (AUG) {
                        lik_partial_aug<T, FINE, NPX>(mu_g, phi_g, Ks, im, i, j, lt, NT, delta, muv, phv, pr2 + twarp * 4,
                                                 lane, false);
                    } else if constexpr (SWIN) {
                        // the speculative copy is stale: copy the window again (every
                        // thread of the team finished reading it before the barrier above)
                        stage_issue(e_cur);
                        stage_wait(sb);
                        lik_partial_staged<RES>(wmu, wcum, wcum2, BW, wdx, dat_s, dat_g, Ks, im, i, j, a_lo, b_lo, rw,
                                                lt, NT, delta, pr2 + twarp * 4, lane);
                    } else {
                        lik_partial<T, RES, CUM, FINE, NPX>(mu_g, cum_g, cum2_g, dat_s, dat_g, Ks, im, i, j, a_lo, b_lo, rw, lt, NT,
                                                 delta, muv, pr2 + twarp * 4, lane, cq, cq2, false);
                    }
                }
                __syncthreads();
                if (SWIN && s_abort) {
                    stage_drain();
                    return;
                }
                if (active) decide();
            }
            // the first round's successor, now that the neighbour wait is over
            if (SANY && r == 0 && rounds > 1) stage_issue(e_cur + 1);
            if (active && nonfin && lt == 0) report_nonfinite(a.err, ch.chain, m, t, (double)dL, (double)dP);
            if (active) {
                if (accept) {
                    const bool one_batch = LL <= NT * NPX;
                    for (int k0 = lt; k0 < LL; k0 += NT * NPX) {
#pragma unroll
                        for (int jj = 0; jj < NPX; ++jj) {
                            const int k = k0 + jj * NT;
                            int aa, bb, kw;
                            if (win_cell<FINE>(im, i, j, k, aa, bb, kw)) {
                                // same value the proposal was scored with: still in registers when
                                // the window took one batch (or in the staged copy), else reloaded
                                // (unchanged since)
                                const size_t idx = (size_t)aa * im.mu_pitch + bb;
                                const int widx = (k / L) * BW + wdx + (k - (k / L) * L);
                                const T old = SWIN ? (T)wmu[widx] : one_batch ? muv[jj] : __ldcg(mu_g + idx);
                                const T xk = mul_rn(delta, Ks[kw]);
                                const T nmu = add_rn(old, xk);
                                __stcg(mu_g + idx, nmu);
                                if (CUM) {
                                    const float d = (float)xk * Prec<float>::rcp((float)old);
                                    Cum6 nq;
                                    if (fabsf(d) <= kCumShift) {
                                        if constexpr (SWIN) nq = cgf_shift(wcum[widx], wcum2[widx], log1p_small(d));
                                        else nq = cgf_shift(__ldcg(cum_g + idx), __ldcg(cum2_g + idx), log1p_small(d));
                                    } else {
                                        const Dat4<T> dv = RES ? dat_s[(aa - a_lo) * rw + (bb - b_lo)] : dat_g[(size_t)aa * W + bb];
                                        nq = photon_cumulants_call((float)nmu, (float)dv.c, (float)dv.is2,
                                                                   (float)dv.beta);
                                    }
                                    __stcg(cum_g + idx, nq.a);
                                    __stcg(cum2_g + idx, nq.b);
                                }
                            }
                        }
                    }
                    for (int e = lt; e < sh.nhalf; e += NT) {
                        T wr, wi;
                        twiddle(tws, sh, ekl[sh.ent_off + e], u, v, wr, wi);
                        spec_p[2 * e] = fma(delta, wr, spec_rd[2 * e]);
                        spec_p[2 * e + 1] = fma(delta, wi, spec_rd[2 * e + 1]);
                    }
                    if (lt == 0) {
                        if (RES) rho_s[(size_t)q * S2 + u * S + v] = r_new;
                        rho_g[m] = r_new;
                        ch.trace_part[(size_t)slot * im.n_patches + pi * im.npj + pj] += (double)dL + (double)dP;
                        ++n_acc;
                        s_acc_any = 1;
                    }
                }
                if (ch.acc_log != nullptr && lt == 0) ch.acc_log[(size_t)(t - 1) * im.Ho * im.Wo + m] = accept ? 1 : 0;
                if (ch.steps != nullptr && t <= im.burn_in && lt == 0) {
                    // burn-in adaptation of the pixel's proposal scale
                    T* sg = reinterpret_cast<T*>(ch.steps);
                    const T sn = sg[m] * (T)im.adapt_fac[2 * (t - 1) + (accept ? 0 : 1)];
                    sg[m] = sn < (T)1e-4 ? (T)1e-4 : sn > (T)4 ? (T)4 : sn;
                }
            }
            if (blk) {
                if (stale || any_accept) __syncthreads();
            } else if (any_accept) {
                tsync();
            }
        }
        // team barriers: the block meets before the sweep's end work and the
        // publish (which must follow both teams' writes), and a team's failed
        // copy wait (s_abort) is acted on here
        if (tb) {
            __syncthreads();
            if (s_abort) {
                stage_drain();
                return;
            }
        }
        if (c == S2 - 1) {
            // a7: after the sweep, add the object to the running sums (own
            // patches only) and, every sample_every-th sweep, keep it
            if (t > im.burn_in) {
                const int ks = t - im.burn_in;
                const int slot_k = (ch.samples != nullptr && ks % im.sample_every == 0) ? ks / im.sample_every - 1 : -1;
                T* keep = slot_k >= 0 && slot_k < im.n_samples
                              ? reinterpret_cast<T*>(ch.samples) + (size_t)slot_k * im.Ho * im.Wo
                              : nullptr;
                for (int q = 0; q < npt; ++q) {
                    const int pi = pi0 + q / tw_, pj = pj0 + (q - (q / tw_) * tw_);
                    const Shape& sh = im.shape[shape_index(im, pi, pj)];
                    for (int e = tid; e < sh.ph * sh.pw; e += blockDim.x) {
                        const int uu = e / sh.pw, vv = e - (e / sh.pw) * sh.pw;
                        const size_t mm = (size_t)(pi * S + uu) * im.Wo + pj * S + vv;
                        const T r = RES ? rho_s[(size_t)q * S2 + uu * S + vv] : rho_g[mm];
                        const double rv = (double)r;
                        ch.rho_sum[mm] += rv;
                        if (ch.rho_sq) ch.rho_sq[mm] += rv * rv;
                        if (keep) keep[mm] = r;
                    }
                }
            }
            if (lt == 0 && in_team && n_acc) atomicAdd(ch.acc_count + (t - 1), (unsigned long long)n_acc);
            n_acc = 0;
            __syncthreads();
        }
        if (tid == 0 && (int)blockIdx.x != a.silent_block) {
            // publish the step count with this step's and the previous step's
            // change marks (read by the neighbours' staleness check), unless the
            // step was published right after its wait (s_pub).  A step without an
            // accepted update wrote nothing the neighbours read, and its own
            // reads were consumed before the barrier, so a relaxed addition
            // suffices; otherwise the addition releases the mu writes
            if (s_pub) {
                s_pub = 0;
            } else if (s_acc_any) {
                s_acc_any = 0;
                const int w = prog_word(s + 1, true, s_chg != 0);
                red_add_release(ch.prog + (size_t)tl * kProgStride, w - s_word);
                s_word = w;
                s_chg = 1;
            } else {
                const int w = prog_word(s + 1, false, s_chg != 0);
                red_add_relaxed(ch.prog + (size_t)tl * kProgStride, w - s_word);
                s_word = w;
                s_chg = 0;
            }
        }
        // the next class step's first round: its windows overlap this step's,
        // so its copy is issued after this step's writes (ordered by the
        // barriers above) and checked against the neighbours after their wait
        if (SANY) stage_issue((cs + 1) * rounds);
    }
    if (SANY) stage_drain();
    // ---- epilogue: resident spectra back to global memory
    if (RES) {
        for (int q = 0; q < npt; ++q) {
            const int pi = pi0 + q / tw_, pj = pj0 + (q - (q / tw_) * tw_);
            const Shape& sh = im.shape[shape_index(im, pi, pj)];
            T* dst = spec_g + 2 * im.patch_off[pi * im.npj + pj];
            for (int e = tid; e < 2 * sh.nhalf; e += blockDim.x) dst[e] = spec_s[(size_t)q * 2 * im.max_nhalf + e];
        }
    }
}

// The sweep kernel's form: tile state resident in shared memory or not,
// augmented sampler or not, object lattice finer than the camera or not.
template <typename T>
const void* sweep_fn(bool res, bool aug, bool fine, bool solo, int stg, bool lean = false)
{
    if constexpr (std::is_same<T, float>::value) {
        if (lean && !aug && !fine && !solo && stg == 0)
            return res ? (const void*)k_sweep<T, true, false, false, false, 0, true>
                       : (const void*)k_sweep<T, false, false, false, false, 0, true>;
        if (solo && res && !fine)
            return aug ? (const void*)k_sweep<T, true, true, false, true> : (const void*)k_sweep<T, true, false, false, true>;
        if (stg == 1 && !aug && !fine && !solo)
            return res ? (const void*)k_sweep<T, true, false, false, false, 1>
                       : (const void*)k_sweep<T, false, false, false, false, 1>;
    }
    if (fine) {
        if (aug) return res ? (const void*)k_sweep<T, true, true, true> : (const void*)k_sweep<T, false, true, true>;
        return res ? (const void*)k_sweep<T, true, false, true> : (const void*)k_sweep<T, false, false, true>;
    }
    if (aug) return res ? (const void*)k_sweep<T, true, true, false> : (const void*)k_sweep<T, false, true, false>;
    return res ? (const void*)k_sweep<T, true, false, false> : (const void*)k_sweep<T, false, false, false>;
}

// Raise a kernel form's dynamic shared-memory limit to at least smem.  The
// limit is kept per kernel function (several form flags can name the same
// function), and it only grows, so launches with smaller plans stay valid.
template <typename T>
cudaError_t ensure_smem_limit(bool res, bool aug, bool fine, bool solo, int stg, size_t smem, bool lean = false)
{
    static std::map<const void*, size_t> limit;
    static std::mutex mu;
    const void* fn = sweep_fn<T>(res, aug, fine, solo, stg, lean);
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = limit[fn];
    if (cur >= smem) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) cur = smem;
    return e;
}

// Cooperative launch (all blocks co-resident, which the neighbour waits
// rely on), through the launch-attribute form so that it can be captured in
// a CUDA graph.
template <typename T>
cudaError_t launch_sweep(const SweepArgs& a, int grid, int threads, size_t smem, cudaStream_t st)
{
    SweepArgs args = a;
    void* kargs[] = {&args};
    const void* fn = sweep_fn<T>(a.resident, a.aug, a.fine, a.solo, a.stage, a.lean);
    cudaError_t e = ensure_smem_limit<T>(a.resident, a.aug, a.fine, a.solo, a.stage, smem, a.lean);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, kargs);
}

// Blocks of the sweep kernel resident per SM for this block size and shared
// memory: the smallest over the forms a plan of this kind may launch -- for a
// one-team plan (solo) its one-team form, else the resident and streamed
// forms (so that either fits), or the staged forms of a staging plan.
template <typename T>
int sweep_blocks_per_sm(int threads, size_t smem, bool aug, bool fine, int stg, bool solo, bool lean)
{
    int best = 1 << 30;
    for (int res = 0; res <= 1; ++res) {
        const bool so = solo && stg == 0;
        if (so && res == 0) continue;   // the one-team form is resident
        int n = 0;
        const bool ln = lean && !so;
        if (ensure_smem_limit<T>(res != 0, aug, fine, so, stg, smem, ln) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_fn<T>(res != 0, aug, fine, so, stg, ln), threads,
                                                          smem) != cudaSuccess)
            return 0;
        best = n < best ? n : best;
    }
    return best;
}

template cudaError_t launch_sweep<float>(const SweepArgs&, int, int, size_t, cudaStream_t);
template cudaError_t launch_sweep<double>(const SweepArgs&, int, int, size_t, cudaStream_t);
template int sweep_blocks_per_sm<float>(int, size_t, bool, bool, int, bool, bool);
template int sweep_blocks_per_sm<double>(int, size_t, bool, bool, int, bool, bool);

// ---------------------------------------------------------------- delta --
// The same per-update arithmetic for one hypothetical proposal (testing):
// one team, the same pixel and entry assignment and reduction order.
template <typename T>
__global__ void __launch_bounds__(256) k_delta(const Image* imp, const Chain* chp, int64_t m, double rho_new, double* out)
{
    using P = Prec<T>;
    __shared__ T red[8][4];
    __shared__ int s_bad;
    const Image& im = *imp;
    const Chain& ch = *chp;
    const int lt = threadIdx.x, lane = lt & 31, twarp = lt >> 5;
    const int NT = im.team, nwt = NT >> 5;
    const int i = (int)(m / im.Wo), j = (int)(m % im.Wo);
    const int S = im.S, W = im.W, LL = im.Lc * im.Lc;
    const int pi = i / S, pj = j / S, u = i - pi * S, v = j - pj * S;
    const Shape& sh = im.shape[shape_index(im, pi, pj)];
    const T* rho = reinterpret_cast<const T*>(ch.rho);
    const T delta = (T)rho_new - rho[m];
    const T* K = kern<T>(im);
    const Dat4<T>* dt = dat<T>(im);
    const T* mu = reinterpret_cast<const T*>(ch.mu);
    const T* spec = reinterpret_cast<const T*>(ch.spec) + 2 * im.patch_off[pi * im.npj + pj];
    if (lt == 0) s_bad = 0;
    bool badP = false, badL = false;
    T accP = 0, accS = 0, accA = 0, accL = 0;
    for (int e = lt; e < sh.nhalf; e += NT) {
        T wr, wi;
        const int ent = sh.ent_off + e;
        twiddle(twid<T>(im), sh, im.ent_kl[ent], u, v, wr, wi);
        prior_term<T>(spec[2 * e], spec[2 * e + 1], wr, wi, delta, ent_wa<T>(im)[ent], ent_m<T>(im)[ent], accP, accS,
                      accA, badP);
    }
    for (int k0 = lt; k0 < LL; k0 += NT * kMaxPx)
        for (int jj = 0; jj < kMaxPx; ++jj) {
            const int k = k0 + jj * NT;
            int aa, bb, kw;
            if (im.f > 1 ? win_cell<true>(im, i, j, k, aa, bb, kw) : win_cell<false>(im, i, j, k, aa, bb, kw)) {
                const size_t idx = (size_t)aa * im.mu_pitch + bb;
                const T xk = mul_rn(delta, K[kw]);
                if (std::is_same<T, float>::value && ch.cum) {
                    const float d = (float)xk * Prec<float>::rcp((float)mu[idx]);
                    if (fabsf(d) <= kCumEval) {
                        accL += (T)cgf_delta((float)xk, log1p_cum(d), ch.cum[idx], ch.cum2[idx]);
                        continue;
                    }
                }
                const Dat4<T> dv = dt[(size_t)aa * W + bb];
                accL += dl_pixel<T>(mu[idx], xk, dv.c, dv.is2, dv.beta, badL);
            }
        }
    accP = warp_sum(accP);
    accS = warp_sum(accS);
    accA = warp_sum(accA);
    accL = warp_sum(accL);
    const bool b = __any_sync(0xffffffffu, badP || badL);
    __syncthreads();
    if (lane == 0) {
        red[twarp][0] = accP;
        red[twarp][1] = accS;
        red[twarp][2] = accA;
        red[twarp][3] = accL;
        if (b) atomicOr(&s_bad, 1);
    }
    __syncthreads();
    if (lt == 0) {
        T sP = 0, sS = 0, sA = 0, sL = 0;
        for (int w = 0; w < nwt; ++w) {
            sP += red[w][0];
            sS += red[w][1];
            sA += red[w][2];
            sL += red[w][3];
        }
        out[0] = (double)sL;
        out[1] = (double)(sP + (T)(sh.K - 1) * P::log1p(sS / sA));
        out[2] = s_bad ? 0.0 : 1.0;
    }
}

template <typename T>
void launch_delta(const Image* d_im, const Chain* d_ch, int64_t m, double rho_new, double* out3, int team,
                  cudaStream_t st, int64_t* launches)
{
    k_delta<T><<<1, team, 0, st>>>(d_im, d_ch, m, rho_new, out3);
    ++*launches;
}
template void launch_delta<float>(const Image*, const Chain*, int64_t, double, double*, int, cudaStream_t, int64_t*);
template void launch_delta<double>(const Image*, const Chain*, int64_t, double, double*, int, cudaStream_t, int64_t*);

}  // namespace bd
