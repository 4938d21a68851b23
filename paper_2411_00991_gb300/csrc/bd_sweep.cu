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
// Per update (one warp, fixed lane assignment => bit-identical results for
// any tiling):
//   a2  Philox4x32-10 counter (m, t, chain, 0) -> z, u; rho' = rho e^{step z}
//   a3  dL = sum over the L x L PSF window of the Eq. 6 change (dl_pixel)
//   a4  dP = patch Dirichlet change (Eq. 7-8) with X'_k = X_k + delta w_k
//   a5  accept iff log u < dL + dP + step z; write rho, mu window, spectrum
//   a7  after the last class of a sweep: running sums of rho (double)
#include <cstdio>

#include "bd_device.cuh"

namespace bd {

template <typename T>
__device__ __forceinline__ void update_pixel(const Image& im, const Chain& ch, int pi, int pj,
                                             int u, int v, int t, int slot, int& n_acc)
{
    using P = Prec<T>;
    using T2 = typename Vec2<T>::type;
    const int lane = threadIdx.x & 31;
    const int sidx = shape_index(im, pi, pj);
    const Shape& sh = im.shape[sidx];
    if (u >= sh.ph || v >= sh.pw) return;   // this class has no pixel in a short patch
    const int S = im.S, L = im.L, R = im.R, H = im.H, W = im.W;
    const int i = pi * S + u, j = pj * S + v;
    const int m = i * im.Wo + j;
    const int p = pi * im.npj + pj;

    // a2: proposal
    const uint4 x = philox4x32_10(make_uint4((uint32_t)m, (uint32_t)t, (uint32_t)ch.chain, 0u),
                                  im.seed_lo, im.seed_hi);
    const T z = P::gauss(uniform23<T>(x.x), uniform23<T>(x.y));
    const T lu = P::log(uniform23<T>(x.z));
    T* rho = reinterpret_cast<T*>(ch.rho);
    const T r_old = rho[m];
    const T step = (T)im.step;
    const T r_new = r_old * P::exp(step * z);
    const T delta = r_new - r_old;

    // a3: likelihood change over the PSF window (camera rows i-2R..i, cols j-2R..j)
    const T* K = kern<T>(im);
    const Dat4<T>* dt = dat<T>(im);
    T* mu = reinterpret_cast<T*>(ch.mu);
    const int a0 = i - 2 * R, b0 = j - 2 * R, LL = L * L;
    const int sdy = 32 / L, sdx = 32 - sdy * L;
    bool bad = false;
    T accL = (T)0;
    {
        int dy = lane / L, dx = lane - (lane / L) * L;
        for (int k = lane; k < LL; k += 32) {
            const int a = a0 + dy, b = b0 + dx;
            if ((unsigned)a < (unsigned)H && (unsigned)b < (unsigned)W) {
                const T xk = mul_rn(delta, __ldg(K + k));
                const T muv = __ldcg(mu + (size_t)a * im.mu_pitch + b);
                const Dat4<T> dv = dt[(size_t)a * W + b];
                accL += dl_pixel<T>(muv, xk, dv.c, dv.is2, dv.beta, bad);
            }
            dx += sdx;
            dy += sdy;
            if (dx >= L) { dx -= L; ++dy; }
        }
    }
    accL = warp_sum(accL);

    // a4: prior change for the patch holding (i, j)
    T2* spec = reinterpret_cast<T2*>(ch.spec) + im.patch_off[p];
    const int* ekl = im.ent_kl + sh.ent_off;
    const T* ewa = ent_wa<T>(im) + sh.ent_off;
    const T* em = ent_m<T>(im) + sh.ent_off;
    const T2* twh = reinterpret_cast<const T2*>(twid<T>(im)) + sh.twh_off;
    const T2* tww = reinterpret_cast<const T2*>(twid<T>(im)) + sh.tww_off;
    T accP = (T)0, accS = (T)0, accA = (T)0;
    for (int e = lane; e < sh.nhalf; e += 32) {
        const int kl = __ldg(ekl + e);
        const int k = kl >> 16, l = kl & 0xffff;
        const T2 eh = twh[(k * u) % sh.ph], ew = tww[(l * v) % sh.pw];
        const T wr = eh.x * ew.x - eh.y * ew.y, wi = eh.x * ew.y + eh.y * ew.x;
        const T2 X = spec[e];
        const T n2 = X.x * X.x + X.y * X.y;
        const T dd = delta * ((T)2 * (X.x * wr + X.y * wi) + delta);   // |X'|^2 - |X|^2
        const T rn = fma(delta, wr, X.x), in = fma(delta, wi, X.y);
        const T n2n = rn * rn + in * in;
        if (!(n2n > (T)0)) bad = true;
        const T mo = P::sqrt(n2), mn = P::sqrt(n2n);
        const T mult = __ldg(em + e);
        accP += __ldg(ewa + e) * P::log1p(dd / n2);
        accS += mult * (dd / (mn + mo));                               // |X'| - |X|
        accA += mult * mo;
    }
    accP = warp_sum(accP);
    accS = warp_sum(accS);
    accA = warp_sum(accA);
    const T dP = accP + (T)(sh.K - 1) * P::log1p(accS / accA);
    bad = __any_sync(0xffffffffu, bad);

    // a5: Metropolis-Hastings test with the Hastings term of the log-space walk
    const bool accept = !bad && (lu < accL + dP + step * z);
    if (accept) {
        int dy = lane / L, dx = lane - (lane / L) * L;
        for (int k = lane; k < LL; k += 32) {
            const int a = a0 + dy, b = b0 + dx;
            if ((unsigned)a < (unsigned)H && (unsigned)b < (unsigned)W) {
                T* q = mu + (size_t)a * im.mu_pitch + b;
                __stcg(q, add_rn(__ldcg(q), mul_rn(delta, __ldg(K + k))));
            }
            dx += sdx;
            dy += sdy;
            if (dx >= L) { dx -= L; ++dy; }
        }
        for (int e = lane; e < sh.nhalf; e += 32) {
            const int kl = __ldg(ekl + e);
            const int k = kl >> 16, l = kl & 0xffff;
            const T2 eh = twh[(k * u) % sh.ph], ew = tww[(l * v) % sh.pw];
            const T wr = eh.x * ew.x - eh.y * ew.y, wi = eh.x * ew.y + eh.y * ew.x;
            T2 X = spec[e];
            X.x = fma(delta, wr, X.x);
            X.y = fma(delta, wi, X.y);
            spec[e] = X;
        }
        if (lane == 0) {
            rho[m] = r_new;
            ch.trace_part[(size_t)slot * im.n_patches + p] += (double)accL + (double)dP;
        }
        ++n_acc;
    }
    if (ch.acc_log != nullptr && lane == 0)
        ch.acc_log[(size_t)(t - 1) * im.Ho * im.Wo + m] = accept ? 1 : 0;
}

template <typename T>
__global__ void __launch_bounds__(256) k_sweep(SweepArgs a)
{
    __shared__ int s_nbr[8];
    __shared__ int s_nn;
    __shared__ int s_abort;
    __shared__ int s_ci;

    // locate this block's chain and tile
    if (threadIdx.x == 0) {
        int lo = 0, hi = a.n_chains - 1;
        while (lo < hi) {   // last chain with cta_base <= blockIdx.x
            const int mid = (lo + hi + 1) >> 1;
            if (a.chains[mid].cta_base <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
        }
        s_ci = lo;
    }
    __syncthreads();
    const Chain& ch = a.chains[s_ci];
    const Image& im = a.imgs[ch.img];
    const int tl = (int)blockIdx.x - ch.cta_base;
    const int ti = tl / ch.ntj, tj = tl - (tl / ch.ntj) * ch.ntj;
    if (threadIdx.x == 0) {
        int nn = 0;
        for (int di = -1; di <= 1; ++di)
            for (int dj = -1; dj <= 1; ++dj) {
                const int ni = ti + di, nj = tj + dj;
                if ((di || dj) && ni >= 0 && ni < ch.nti && nj >= 0 && nj < ch.ntj)
                    s_nbr[nn++] = ni * ch.ntj + nj;
            }
        s_nn = nn;
        s_abort = 0;
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int pi0 = ti * ch.tpi, pj0 = tj * ch.tpj;
    const int pi1 = min(pi0 + ch.tpi, im.npi), pj1 = min(pj0 + ch.tpj, im.npj);
    const int tw_ = pj1 - pj0, npt = (pi1 - pi0) * tw_;
    const int S = im.S, S2 = S * S;
    const int nsteps = a.n_sweeps * S2;
    int n_acc = 0;

    for (int s = 0; s < nsteps; ++s) {
        const int slot = s / S2, c = s - slot * S2;
        const int t = a.t0 + 1 + slot;
        const int u = c / S, v = c - (c / S) * S;
        if (s > 0) {
            if (warp == 0) {
                const bool ok = warp_wait_flags(ch.prog, s_nbr, s_nn, s, a.err);
                if (lane == 0 && !ok) s_abort = 1;
            }
            __syncthreads();
            if (s_abort) return;
        }
        for (int q = warp; q < npt; q += nw) {
            const int pi = pi0 + q / tw_, pj = pj0 + (q - (q / tw_) * tw_);
            update_pixel<T>(im, ch, pi, pj, u, v, t, slot, n_acc);
        }
        if (c == S2 - 1) {
            __syncwarp();
            // a7: after the sweep, add the object to the running sums (own patches only)
            if (t > im.burn_in) {
                const T* rho = reinterpret_cast<const T*>(ch.rho);
                for (int q = warp; q < npt; q += nw) {
                    const int pi = pi0 + q / tw_, pj = pj0 + (q - (q / tw_) * tw_);
                    const Shape& sh = im.shape[shape_index(im, pi, pj)];
                    for (int e = lane; e < sh.ph * sh.pw; e += 32) {
                        const int uu = e / sh.pw, vv = e - (e / sh.pw) * sh.pw;
                        const size_t mm = (size_t)(pi * S + uu) * im.Wo + pj * S + vv;
                        const double rv = (double)rho[mm];
                        ch.rho_sum[mm] += rv;
                        if (ch.rho_sq) ch.rho_sq[mm] += rv * rv;
                    }
                }
            }
            if (lane == 0 && n_acc) atomicAdd(ch.acc_count + (t - 1), (unsigned long long)n_acc);
            n_acc = 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            st_release(ch.prog + tl, s + 1);
        }
    }
}

template <typename T>
cudaError_t launch_sweep(const SweepArgs& a, int grid, int warps, cudaStream_t st)
{
    SweepArgs args = a;
    void* kargs[] = {&args};
    return cudaLaunchCooperativeKernel((const void*)k_sweep<T>, dim3(grid), dim3(32 * warps), kargs,
                                       0, st);
}

template <typename T>
int sweep_blocks_per_sm(int warps)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<T>, 32 * warps, 0) != cudaSuccess)
        return 0;
    return n;
}

template cudaError_t launch_sweep<float>(const SweepArgs&, int, int, cudaStream_t);
template cudaError_t launch_sweep<double>(const SweepArgs&, int, int, cudaStream_t);
template int sweep_blocks_per_sm<float>(int);
template int sweep_blocks_per_sm<double>(int);

// ---------------------------------------------------------------- delta --
// The same per-update arithmetic for one hypothetical proposal (testing).
template <typename T>
__global__ void k_delta(const Image* imp, const Chain* chp, int64_t m, double rho_new, double* out)
{
    using P = Prec<T>;
    using T2 = typename Vec2<T>::type;
    const Image& im = *imp;
    const Chain& ch = *chp;
    const int lane = threadIdx.x & 31;
    const int i = (int)(m / im.Wo), j = (int)(m % im.Wo);
    const int S = im.S, L = im.L, R = im.R, H = im.H, W = im.W;
    const int pi = i / S, pj = j / S, u = i - pi * S, v = j - pj * S;
    const int p = pi * im.npj + pj;
    const Shape& sh = im.shape[shape_index(im, pi, pj)];
    const T* rho = reinterpret_cast<const T*>(ch.rho);
    const T delta = (T)rho_new - rho[m];
    const T* K = kern<T>(im);
    const Dat4<T>* dt = dat<T>(im);
    const T* mu = reinterpret_cast<const T*>(ch.mu);
    bool bad = false;
    T accL = (T)0;
    for (int k = lane; k < L * L; k += 32) {
        const int a = i - 2 * R + k / L, b = j - 2 * R + k % L;
        if ((unsigned)a < (unsigned)H && (unsigned)b < (unsigned)W) {
            const Dat4<T> dv = dt[(size_t)a * W + b];
            accL += dl_pixel<T>(mu[(size_t)a * im.mu_pitch + b], mul_rn(delta, K[k]), dv.c, dv.is2, dv.beta, bad);
        }
    }
    accL = warp_sum(accL);
    const T2* spec = reinterpret_cast<const T2*>(ch.spec) + im.patch_off[p];
    const T2* twh = reinterpret_cast<const T2*>(twid<T>(im)) + sh.twh_off;
    const T2* tww = reinterpret_cast<const T2*>(twid<T>(im)) + sh.tww_off;
    T accP = (T)0, accS = (T)0, accA = (T)0;
    for (int e = lane; e < sh.nhalf; e += 32) {
        const int kl = im.ent_kl[sh.ent_off + e];
        const int k = kl >> 16, l = kl & 0xffff;
        const T2 eh = twh[(k * u) % sh.ph], ew = tww[(l * v) % sh.pw];
        const T wr = eh.x * ew.x - eh.y * ew.y, wi = eh.x * ew.y + eh.y * ew.x;
        const T2 X = spec[e];
        const T n2 = X.x * X.x + X.y * X.y;
        const T dd = delta * ((T)2 * (X.x * wr + X.y * wi) + delta);
        const T rn = fma(delta, wr, X.x), in = fma(delta, wi, X.y);
        const T n2n = rn * rn + in * in;
        if (!(n2n > (T)0)) bad = true;
        const T mo = P::sqrt(n2), mn = P::sqrt(n2n);
        const T mult = ent_m<T>(im)[sh.ent_off + e];
        accP += ent_wa<T>(im)[sh.ent_off + e] * P::log1p(dd / n2);
        accS += mult * (dd / (mn + mo));
        accA += mult * mo;
    }
    accP = warp_sum(accP);
    accS = warp_sum(accS);
    accA = warp_sum(accA);
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
        out[0] = (double)accL;
        out[1] = (double)(accP + (T)(sh.K - 1) * P::log1p(accS / accA));
        out[2] = bad ? 0.0 : 1.0;
    }
}

template <typename T>
void launch_delta(const Image* d_im, const Chain* d_ch, int64_t m, double rho_new, double* out3,
                  cudaStream_t st, int64_t* launches)
{
    k_delta<T><<<1, 32, 0, st>>>(d_im, d_ch, m, rho_new, out3);
    ++*launches;
}
template void launch_delta<float>(const Image*, const Chain*, int64_t, double, double*, cudaStream_t, int64_t*);
template void launch_delta<double>(const Image*, const Chain*, int64_t, double, double*, cudaStream_t, int64_t*);

}  // namespace bd
