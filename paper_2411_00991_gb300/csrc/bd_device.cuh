// bd_device.cuh -- device helpers of the libbdecon kernels: Philox4x32-10,
// precision traits, warp reductions, flag waits, and the per-pixel
// likelihood change of Eq. 6 written as a ratio of photon-count sums.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <math_constants.h>

#include "bd_internal.h"

namespace bd {

// ---------------------------------------------------------------- Philox --
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit multiplies with Weyl-sequence key increments.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// ((x >> 9) + 1/2) * 2^-23: 24 significant bits, exact in float and double.
template <typename T>
__device__ __forceinline__ T uniform23(uint32_t x)
{
    return ((T)(x >> 9) + (T)0.5) * (T)1.1920928955078125e-07;
}

// ------------------------------------------------------ precision traits --
template <typename T> struct Prec;

template <> struct Prec<float> {
    static constexpr float kEps = 1.4901161193847656e-08f;  // 2^-26: sum truncation
    static constexpr float kMaxExp = 80.0f;
    static constexpr float kMaxFinite = 3.4028234663852886e38f;
    static __device__ __forceinline__ float log(float x) { return logf(x); }
    static __device__ __forceinline__ float exp(float x) { return expf(x); }
    static __device__ __forceinline__ float log1p(float x) { return log1pf(x); }
    static __device__ __forceinline__ float sqrt(float x) { return sqrtf(x); }
    // photon-weight scale factors only shift relative term weights, which
    // cancel to first order in the ratio; fast intrinsics suffice there
    static __device__ __forceinline__ float wlog(float x) { return __logf(x); }
    static __device__ __forceinline__ float wexp(float x) { return __expf(x); }
    static __device__ __forceinline__ float rcp(float x)
    {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    static __device__ __forceinline__ float gauss(float u0, float u1)
    {
        return sqrtf(-2.0f * logf(u0)) * cospif(2.0f * u1);
    }
};

template <> struct Prec<double> {
    static constexpr double kEps = 1.3877787807814457e-17;  // 2^-56
    static constexpr double kMaxExp = 700.0;
    static constexpr double kMaxFinite = 1.7976931348623157e308;
    static __device__ __forceinline__ double log(double x) { return ::log(x); }
    static __device__ __forceinline__ double exp(double x) { return ::exp(x); }
    static __device__ __forceinline__ double log1p(double x) { return ::log1p(x); }
    static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
    static __device__ __forceinline__ double wlog(double x) { return ::log(x); }
    static __device__ __forceinline__ double wexp(double x) { return ::exp(x); }
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double gauss(double u0, double u1)
    {
        return ::sqrt(-2.0 * ::log(u0)) * ::cos(2.0 * CUDART_PI * u1);
    }
};

// Explicitly rounded product and sum (never contracted into an FMA), so the
// expected-image value a proposal is scored with is bit-identical to the
// value written when it is accepted.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

template <typename T> struct alignas(4 * sizeof(T)) Dat4 { T c, is2, beta, lnorm; };

template <typename T> __device__ __forceinline__ const T* kern(const Image& im);
template <> __device__ __forceinline__ const float* kern<float>(const Image& im) { return im.Ke32; }
template <> __device__ __forceinline__ const double* kern<double>(const Image& im) { return im.Ke64; }
template <typename T> __device__ __forceinline__ const Dat4<T>* dat(const Image& im);
template <> __device__ __forceinline__ const Dat4<float>* dat<float>(const Image& im)
{
    return reinterpret_cast<const Dat4<float>*>(im.dat32);
}
template <> __device__ __forceinline__ const Dat4<double>* dat<double>(const Image& im)
{
    return reinterpret_cast<const Dat4<double>*>(im.dat64);
}
template <typename T> __device__ __forceinline__ const T* ent_wa(const Image& im);
template <> __device__ __forceinline__ const float* ent_wa<float>(const Image& im) { return im.ent_wa32; }
template <> __device__ __forceinline__ const double* ent_wa<double>(const Image& im) { return im.ent_wa64; }
template <typename T> __device__ __forceinline__ const T* ent_m(const Image& im);
template <> __device__ __forceinline__ const float* ent_m<float>(const Image& im) { return im.ent_m32; }
template <> __device__ __forceinline__ const double* ent_m<double>(const Image& im) { return im.ent_m64; }
template <typename T> __device__ __forceinline__ const T* twid(const Image& im);
template <> __device__ __forceinline__ const float* twid<float>(const Image& im) { return im.tw32; }
template <> __device__ __forceinline__ const double* twid<double>(const Image& im) { return im.tw64; }

// ------------------------------------------------------------ warp sums --
template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Barrier of the n threads (whole warps) of one of two update teams: named
// barrier 1 or 2 (0 is the block-wide barrier of __syncthreads).  Orders the
// team's shared- and global-memory accesses like __syncthreads does for the
// block.  The ids are immediates, so a kernel reserves three barriers, not
// the sixteen that an id held in a register would reserve (which costs
// resident blocks per SM).
__device__ __forceinline__ void team_bar2(int team, int n)
{
    if (team == 0) asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory");
    else asm volatile("bar.sync 2, %0;" ::"r"(n) : "memory");
}

// ------------------------------------------------------ memory ordering --
// Fire-and-forget additions to a progress word.  Publishing by read-modify-
// write keeps every word a reader can observe in observation order after the
// tile's last release (PTX memory model: observation order runs through
// atomic read-modify-writes, not plain stores), so a reader's acquire
// synchronises with the tile's last change whatever later word it reads.
__device__ __forceinline__ void red_add_release(int* p, int v)
{
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_add_relaxed(int* p, int v)
{
    asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed(const int* p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void fence_acq_rel_gpu()
{
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Progress word of a tile: (steps published << 2) | c0 | c1 << 1, c0 (c1)
// set when the tile changed data its neighbours' windows read (an accepted
// update, or the photon counts) at the last (the one before the last)
// published step.  One word carries both the step count a neighbour waits
// for and what it needs to know whether its speculative score went stale.
__device__ __forceinline__ int prog_word(int steps, bool changed, bool changed_before)
{
    return (steps << 2) | (changed ? 1 : 0) | (changed_before ? 2 : 0);
}

// Bounded wait of one warp until every neighbour nbr[i] (i < nn, one per
// lane) has published at least `need` steps.  Gives up (setting kErrTimeout)
// after wait_ns nanoseconds (default 4 s) or 2^26 polls, or as soon as any
// other block has raised an error.  Returns true if every flag arrived; word
// receives the lane's neighbour word as the wait saw it (relaxed: the caller
// follows the wait with fence_acq_rel_gpu, by every lane, where it reads
// data the neighbours wrote).  pre: the word as this lane read it earlier
// (relaxed), 0 if none; when it already shows the step, no load is issued.
constexpr uint64_t kWaitNs = 4000000000ull;
constexpr uint32_t kWaitPolls = 1u << 26;
__device__ __forceinline__ bool warp_wait_flags(const int* prog, const int* nbr, int nn, int need,
                                                int* err, uint64_t wait_ns, int& word, int pre = 0)
{
    const int lane = threadIdx.x & 31;
    bool ok = true;
    word = 0;
    if (lane < nn) {
        const int* f = prog + (size_t)nbr[lane] * kProgStride;
        // poll with relaxed loads (tight for the first polls, then with a short
        // sleep)
        int v = pre;
        if ((v >> 2) < need) v = ld_relaxed(f);
        if ((v >> 2) < need) {
            const uint64_t t0 = global_ns();
            uint32_t it = 0;
            while (((v = ld_relaxed(f)) >> 2) < need) {
                ++it;
                if ((it & 31u) == 0u) {
                    if (ld_relaxed(err) != 0) { ok = false; break; }
                    if (global_ns() - t0 > wait_ns || it > kWaitPolls) {
                        atomicOr(err, kErrTimeout);
                        ok = false;
                        break;
                    }
                }
                if (it > 64u) __nanosleep(32);
            }
        }
        if (ok) word = v;
    }
    return __all_sync(0xffffffffu, ok);
}

// ------------------------------------------- bulk copies (TMA engine) --
// Global -> shared copies issued to the tensor memory accelerator as
// untiled bulk copies (cp.async.bulk), completing on a shared-memory
// mbarrier that counts the bytes still to land.  Both addresses must be
// 16-byte aligned and the size a multiple of 16 bytes; the callers copy
// rows of 16- or 32-byte records between 16-byte-aligned bases.
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    // make the initialised barrier visible to the async proxy that completes it
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// Tiled 2-D copy of one box of a tensor (described by a TMA tensor map in
// global memory, 64-byte aligned) at element coordinates (x, y) into shared
// memory (128-byte aligned), completing on the mbarrier.  x times the
// element size must be a multiple of 16 bytes; y may be negative or past the
// end (those rows, like out-of-range columns, are filled with zeros).
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int x, int y, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
// Orders this thread's earlier generic-proxy accesses to global memory (and
// those made visible to it by barriers and acquire fences) before its later
// async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// Bounded wait for phase `parity` of the barrier to complete: false after
// wait_ns nanoseconds or 2^26 tries.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t wait_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1; it <= kWaitPolls; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0u && global_ns() - t0 > wait_ns) break;
    }
    return false;
}

// ------------------------------------------- photon-count augmentation --
// Draw of a photon count from p(phi | w, mu) ∝ exp(-(c - phi)^2 is2 / 2)
// mu^phi / phi!  (the summands of Eq. 6: Normal(w; G phi + o, var) times
// Poisson(phi; mu), in photon units) by inverse CDF at u.  With
// g(phi) = log(T_{phi+1} / T_phi) = is2 (c - phi - 1/2) + log mu - log(phi + 1),
// decreasing in phi (the summand is log-concave), the integer mode is reached
// by stepping from the Gaussian-approximation centre; terms relative to the
// mode are kept while above 2^-60 of it (double) or 2^-30 (float), and the
// cumulative weight is summed upward from the lowest kept count.  Sets
// status when a walk would exceed kPhiSteps terms.
constexpr int kPhiSteps = 1 << 16;

template <typename T>
__device__ __forceinline__ int sample_phi(T mu, T c, T is2, T u, int& status)
{
    using P = Prec<T>;
    const T lmu = P::log(mu);
    const T cut = sizeof(T) == 8 ? (T)(-60.0 * 0.69314718055994531) : (T)(-30.0 * 0.69314718055994531);
    T f0 = mu * (c * is2 + (T)1) / (mu * is2 + (T)1);
    f0 = f0 < (T)1.0e7 ? f0 : (T)1.0e7;
    int m = f0 > (T)0 ? (int)f0 : 0;
    int it = 0;
#define BD_G(f) (is2 * (c - (T)(f) - (T)0.5) + lmu - P::log((T)((f) + 1)))
    while (BD_G(m) > (T)0 && it < kPhiSteps) { ++m; ++it; }
    while (m > 0 && BD_G(m - 1) < (T)0 && it < kPhiSteps) { --m; ++it; }
    T Z = (T)1, l = (T)0, llo = (T)0;
    int lo = m, hi = m;
    for (int f = m - 1; f >= 0 && it < kPhiSteps; --f, ++it) {   // log T_f - log T_m
        l -= BD_G(f);
        if (l < cut) break;
        Z += P::exp(l);
        lo = f;
        llo = l;
    }
    l = (T)0;
    for (int f = m; it < kPhiSteps; ++f, ++it) {                  // log T_{f+1} - log T_m
        l += BD_G(f);
        if (l < cut) break;
        Z += P::exp(l);
        hi = f + 1;
    }
    if (it >= kPhiSteps) status = 1;
    const T target = u * Z;
    T acc = (T)0;
    l = llo;
    for (int f = lo; f < hi; ++f) {
        acc += P::exp(l);
        if (acc >= target) return f;
        l += BD_G(f);
    }
#undef BD_G
    return hi;
}

// phi-dependent part of the log completed likelihood of one pixel (Eq. 5):
// -(c - phi)^2 is2 / 2 + phi log mu - log phi!
__device__ __forceinline__ double phi_logterm(int phi, double lmu, double c, double is2)
{
    const double d = c - (double)phi;
    return -0.5 * d * d * is2 + (double)phi * lmu - lgamma((double)phi + 1.0);
}

// Integer mode estimate of the photon posterior (log-concave in phi): the
// Gaussian-approximation centre mu (c + s^2) / (mu + s^2), then one Newton
// step on d/dphi log T_phi ~ (c - phi)/s^2 + log(mu / (phi + 1/2)).  Any
// estimate gives the same sums (they run outward until the terms vanish);
// a close one keeps them short.
__device__ __forceinline__ int photon_mode(float muf, float cf, float isf)
{
    float ph = muf * __fdividef(cf * isf + 1.0f, muf * isf + 1.0f);
    ph = fmaxf(ph, 0.0f);
    const float f = (cf - ph) * isf + __logf(__fdividef(muf, ph + 0.5f));
    const float fp = -isf - __fdividef(1.0f, ph + 0.5f);
    const float phs = fminf(fmaxf(ph - __fdividef(f, fp), 0.0f), 1.0e7f);
    return __float2int_rn(phs);
}

// ---------------------------------------------- per-pixel likelihood change
// Change of the log marginal likelihood of one camera pixel (Eq. 6),
//   l(mu') - l(mu) = -(mu' - mu) + log S(mu') - log S(mu),
//   S(mu) = sum_phi exp(-(c - phi)^2 / (2 s^2)) mu^phi / phi!,
// with c = (w - o)/G and s^2 = var/G^2 (the photon-count form of
// Normal(w; G phi + o, var)).  Writing r = mu'/mu and T_phi for the summand
// at mu, S(mu')/S(mu) = r^phi0 * (B + D)/B with B = sum_phi T_phi and
// D = sum_phi T_phi (r^(phi - phi0) - 1), so
//   l(mu') - l(mu) = -x + phi0 log1p(x/mu) + log1p(D/B),     x = mu' - mu,
// free of cancellation for small x.  The summand is log-concave in phi; the
// sums run outward from phi0 (a Newton estimate of the mode) with term
// ratios updated multiplicatively (the Gaussian factor by exp(-1/s^2) per
// step) until terms fall below kEps of the running sum.
template <typename T>
__device__ __forceinline__ T dl_pixel(T mu, T x, T c, T is2, T beta, bool& bad)
{
    using P = Prec<T>;
    const T mup = add_rn(mu, x);
    if (!(mup > (T)0)) {
        bad = true;
        return (T)0;
    }
    // mode of the photon posterior: Gaussian-approximation centre, then one
    // Newton step on d/dphi log T_phi ~ (c - phi)/s^2 + log(mu / (phi + 1/2))
    const int p0 = photon_mode((float)mu, (float)c, (float)is2);
    const T fp0 = (T)p0;

    const T inv_mu = P::rcp(mu);
    const T d = x * inv_mu;              // r - 1
    const T r = (T)1 + d;
    const T lmu = P::wlog(mu);
    T B = (T)1, D = (T)0;
    // upward: T_{phi+1} = T_phi * mu exp((c - phi - 1/2)/s^2) / (phi + 1);
    // two terms per pass, one exit test per pass (a term below kEps of the
    // sum changes nothing)
    {
        T mg = P::wexp(fmin(lmu + (c - fp0 - (T)0.5) * is2, (T)P::kMaxExp));
        T t = (T)1, e = (T)0;
        T fphi = fp0;
        for (int it = 0; it < 2048; ++it) {
            const T f1 = mg * P::rcp(fphi + (T)1);
            const T f2 = mg * beta * P::rcp(fphi + (T)2);
            fphi += (T)2;
            mg *= beta * beta;
            t *= f1;
            e = fma(e, r, d);                 // r^k - 1
            B += t;
            D = fma(t, e, D);
            t *= f2;
            e = fma(e, r, d);
            B += t;
            D = fma(t, e, D);
            if (t * fmax((T)1, (T)1 + e) < (T)P::kEps * B) break;
        }
    }
    // downward: T_{phi-1} = T_phi * phi exp(-(c - phi + 1/2)/s^2) / mu
    if (p0 > 0) {
        T hq = P::wexp(fmin(-lmu - (c - fp0 + (T)0.5) * is2, (T)P::kMaxExp));
        const T ri = P::rcp(r);
        const T di = -d * ri;                // 1/r - 1
        T t = (T)1, e = (T)0;
        T fphi = fp0;
        int phi = p0;
        for (; phi > 1; phi -= 2) {
            const T f1 = hq * fphi;
            const T f2 = hq * beta * (fphi - (T)1);
            hq *= beta * beta;
            fphi -= (T)2;
            t *= f1;
            e = fma(e, ri, di);               // r^-k - 1
            B += t;
            D = fma(t, e, D);
            t *= f2;
            e = fma(e, ri, di);
            B += t;
            D = fma(t, e, D);
            if (t * fmax((T)1, (T)1 + e) < (T)P::kEps * B) break;
        }
        if (phi == 1) {                       // odd remainder: the phi = 0 term
            t *= hq * fphi;
            e = fma(e, ri, di);
            B += t;
            D = fma(t, e, D);
        }
    }
    return -x + fp0 * P::log1p(d) + P::log1p(D * P::rcp(B));
}

// ------------------------------------------ photon-posterior cumulant cache
// For the float sweep each camera pixel caches the first six cumulants of
// its photon-count posterior w_phi ∝ exp(-(c - phi)^2/(2 s^2)) mu^phi / phi!
// at the current mu, stored as c_j = kappa_j / j! ({c1..c4} and {c5, c6}).
// Since S(mu e^t)/S(mu) = E_w[e^{t phi}], the change of Eq. 6 for
// mu -> mu (1 + d) is -mu d + K(t), t = log1p(d), with K the cumulant
// generating function: K(t) = sum_j c_j t^j.  Window pixels with
// |d| <= kCumEval use the six-term series (the first omitted term,
// kappa7 |t|^7 / 7!, stays below ~5e-8 for photon counts up to ~10^2);
// others use the exact sum (dl_pixel).  When mu changes by an accepted
// update the cache is moved by exponential tilting (the tilted
// distribution's cumulants are the derivatives of K at t:
// c_j' = sum_i C(j+i, i) c_{j+i} t^i) when |d| <= kCumShift, or recomputed
// exactly; the double refresh rebuilds it from scratch.
constexpr float kCumEval = 0.15f;
constexpr float kCumShift = 0.02f;

struct Cum6 {
    float4 a;   // c1 (mean), c2, c3, c4
    float2 b;   // c5, c6
};

// log1p(d): its series to d^5 for |d| <= 0.05 (remainder below d^6/6),
// the library function beyond
__device__ __forceinline__ float log1p_small(float d)
{
    return d * fmaf(d, fmaf(d, fmaf(d, fmaf(d, 0.2f, -0.25f), 0.33333334f), -0.5f), 1.0f);
}
__device__ __forceinline__ float log1p_cum(float d)
{
    return fabsf(d) <= 0.05f ? log1p_small(d) : log1pf(d);
}

// K(t) - x
__device__ __forceinline__ float cgf_delta(float x, float t, float4 a, float2 b)
{
    const float p = fmaf(t, fmaf(t, fmaf(t, fmaf(t, fmaf(t, b.y, b.x), a.w), a.z), a.y), a.x);
    return fmaf(t, p, -x);
}

__device__ __forceinline__ Cum6 cgf_shift(float4 a, float2 b, float t)
{
    Cum6 r;
    r.a.x = fmaf(t, fmaf(t, fmaf(t, fmaf(t, fmaf(t, 6.0f * b.y, 5.0f * b.x), 4.0f * a.w), 3.0f * a.z), 2.0f * a.y), a.x);
    r.a.y = fmaf(t, fmaf(t, fmaf(t, fmaf(t, 15.0f * b.y, 10.0f * b.x), 6.0f * a.w), 3.0f * a.z), a.y);
    r.a.z = fmaf(t, fmaf(t, fmaf(t, 20.0f * b.y, 10.0f * b.x), 4.0f * a.w), a.z);
    r.a.w = fmaf(t, fmaf(t, 15.0f * b.y, 5.0f * b.x), a.w);
    r.b.x = fmaf(t, 6.0f * b.y, b.x);
    r.b.y = b.y;
    return r;
}

// Exact cumulants of the photon posterior at mu (same mode estimate and
// outward recurrences as dl_pixel): raw moments of k = phi - phi0, then
// central moments about the mean, then cumulants.
template <typename T>
__device__ __forceinline__ Cum6 photon_cumulants(T mu, T c, T is2, T beta)
{
    using P = Prec<T>;
    const int p0 = photon_mode((float)mu, (float)c, (float)is2);
    const T fp0 = (T)p0;
    const T lmu = P::wlog(mu);
    T S[7] = {1, 0, 0, 0, 0, 0, 0};
    {
        T mg = P::wexp(fmin(lmu + (c - fp0 - (T)0.5) * is2, (T)P::kMaxExp));
        T t = 1, fphi = fp0, k = 0;
        for (int it = 0; it < 4096; ++it) {
            fphi += (T)1;
            k += (T)1;
            t *= mg * P::rcp(fphi);
            mg *= beta;
            T tk = t;
#pragma unroll
            for (int jj = 0; jj < 7; ++jj) {
                S[jj] += tk;
                tk *= k;
            }
            if (t < (T)P::kEps * (T)0.0625 * S[0]) break;
        }
    }
    if (p0 > 0) {
        T hq = P::wexp(fmin(-lmu - (c - fp0 + (T)0.5) * is2, (T)P::kMaxExp));
        T t = 1, fphi = fp0, k = 0;
        for (int phi = p0; phi > 0; --phi) {
            t *= hq * fphi;
            hq *= beta;
            fphi -= (T)1;
            k -= (T)1;
            T tk = t;
#pragma unroll
            for (int jj = 0; jj < 7; ++jj) {
                S[jj] += tk;
                tk *= k;
            }
            if (t < (T)P::kEps * (T)0.0625 * S[0]) break;
        }
    }
    const T i0 = (T)1 / S[0];
    const T m = S[1] * i0, e2 = S[2] * i0, e3 = S[3] * i0, e4 = S[4] * i0, e5 = S[5] * i0, e6 = S[6] * i0;
    const T m2 = m * m, m3 = m2 * m, m4 = m3 * m;
    const T u2 = e2 - m2;
    const T u3 = e3 - (T)3 * m * e2 + (T)2 * m3;
    const T u4 = e4 - (T)4 * m * e3 + (T)6 * m2 * e2 - (T)3 * m4;
    const T u5 = e5 - (T)5 * m * e4 + (T)10 * m2 * e3 - (T)10 * m3 * e2 + (T)4 * m4 * m;
    const T u6 = e6 - (T)6 * m * e5 + (T)15 * m2 * e4 - (T)20 * m3 * e3 + (T)15 * m4 * e2 - (T)5 * m4 * m2;
    const T k4 = u4 - (T)3 * u2 * u2;
    const T k5 = u5 - (T)10 * u3 * u2;
    const T k6 = u6 - (T)15 * u4 * u2 - (T)10 * u3 * u3 + (T)30 * u2 * u2 * u2;
    Cum6 r;
    r.a = make_float4((float)(fp0 + m), (float)(u2 / (T)2), (float)(u3 / (T)6), (float)(k4 / (T)24));
    r.b = make_float2((float)(k5 / (T)120), (float)(k6 / (T)720));
    return r;
}

// Out-of-line copies for the float sweep, where the exact sums are the rare
// branch: keeping them out of the unrolled window loop keeps register use low.
__device__ __forceinline__ float dl_pixel_call(float mu, float x, float c, float is2, float beta, int* bad)
{
    bool b = false;
    const float r = dl_pixel<float>(mu, x, c, is2, beta, b);
    if (b) *bad = 1;
    return r;
}
__device__ __forceinline__ Cum6 photon_cumulants_call(float mu, float c, float is2, float beta)
{
    return photon_cumulants<float>(mu, c, is2, beta);
}

// Full log marginal likelihood of one camera pixel in double (Eq. 6):
//   l(mu) = -log(2 pi var)/2 - mu + log sum_phi exp(-(c-phi)^2/(2 s^2)) mu^phi / phi!
// evaluated as log T_phi0 + log(sum_phi T_phi / T_phi0) with the same
// outward recurrences (truncation 2^-56).
__device__ __forceinline__ double loglik64(double mu, double c, double is2, double beta,
                                           double lnorm)
{
    const float muf = (float)mu, cf = (float)c, isf = (float)is2;
    float ph = muf * (cf * isf + 1.0f) / (muf * isf + 1.0f);
    ph = fmaxf(ph, 0.0f);
    const float f = (cf - ph) * isf + __logf(muf / (ph + 0.5f));
    const float fp = -isf - 1.0f / (ph + 0.5f);
    const float phs = fminf(fmaxf(ph - f / fp, 0.0f), 1.0e7f);
    const int p0 = __float2int_rn(phs);
    const double fp0 = (double)p0;
    const double lmu = ::log(mu);
    const double lt0 = -0.5 * (c - fp0) * (c - fp0) * is2 + fp0 * lmu - ::lgamma(fp0 + 1.0);
    double B = 1.0;
    {
        double mg = ::exp(fmin(lmu + (c - fp0 - 0.5) * is2, 700.0));
        double t = 1.0, fphi = fp0;
        for (int it = 0; it < 4096; ++it) {
            fphi += 1.0;
            t *= mg / fphi;
            mg *= beta;
            B += t;
            if (t < 1.3877787807814457e-17 * B) break;
        }
    }
    if (p0 > 0) {
        double hq = ::exp(fmin(-lmu - (c - fp0 + 0.5) * is2, 700.0));
        double t = 1.0, fphi = fp0;
        for (int phi = p0; phi > 0; --phi) {
            t *= hq * fphi;
            hq *= beta;
            fphi -= 1.0;
            B += t;
            if (t < 1.3877787807814457e-17 * B) break;
        }
    }
    return lnorm - mu + lt0 + ::log(B);
}

// Patch shape index of patch (pi, pj): bit 1 = partial rows, bit 0 = partial columns.
__device__ __forceinline__ int shape_index(const Image& im, int pi, int pj)
{
    return ((pi + 1) * im.S > im.Ho ? 2 : 0) | ((pj + 1) * im.S > im.Wo ? 1 : 0);
}

}  // namespace bd
