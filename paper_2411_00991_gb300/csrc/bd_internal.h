// bd_internal.h -- device-visible descriptors shared by the libbdecon kernels
// and the host code that builds them.  Nothing here is part of the C ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bd {

constexpr int kMaxShapes = 4;       // patch shapes: full, right, bottom, corner
constexpr int kMaxL = 63;           // largest PSF side
constexpr int kMaxS = 64;           // largest stride (prior patch side)
constexpr int kMaxSlots = 64;       // sweeps per sweep-kernel launch
constexpr int kRedThreads = 256;    // fixed block size of every reduction

// device error flag bits
constexpr int kErrTimeout = 1;
constexpr int kErrNumeric = 2;
constexpr int kErrRatio = 4;        // a proposal's log acceptance ratio was not finite (record in err[1..9])

// One patch shape (ph x pw) of a problem.  The prior of Eq. 8 is evaluated on
// a canonical half of the frequencies: one representative of each Hermitian
// pair {k, -k} with multiplicity 2, self-conjugate frequencies with 1.
struct Shape {
    int ph, pw, K, nhalf;
    int ent_off;            // first entry in the problem's entry arrays
    int twh_off, tww_off;   // twiddle tables exp(-2 pi i j / ph), exp(-2 pi i j / pw)
    float inv_ph, inv_pw;   // 1/ph, 1/pw for the small-integer modulo of twiddle indices
};

// One problem (frame + calibration + PSF), shared by its chains.
struct Image {
    int H, W, L, R, S, Ho, Wo, npi, npj;
    int mu_pitch;                    // elements per row of mu (multiple of 4)
    int n_chains;
    uint32_t seed_lo, seed_hi;
    double step;
    int burn_in, refresh_every;
    int n_patches;
    int chain0;                      // index of its first chain in the chain table
    const double* K64;               // L*L, normalised
    const float* K32;
    const double* dat64;             // per camera pixel {c, 1/s^2, exp(-1/s^2), -log(2 pi var)/2}
    const float* dat32;
    Shape shape[kMaxShapes];
    const int* ent_kl;               // (k << 16) | l
    const double* ent_wa64;          // mult * (alpha - 1) / 2
    const double* ent_m64;           // mult
    const float* ent_wa32;
    const float* ent_m32;
    const double* tw64;              // complex pairs
    const float* tw32;
    const int64_t* patch_off;        // offset (complex elements) of each patch's half spectrum
    int64_t spec_len;                // complex elements per chain
    int n_ent, n_tw, max_nhalf;      // table sizes (all shapes)
    int team;                        // threads per pixel update (a property of the problem)
    int f, Le, Lc;                   // object cells per camera pixel side, effective kernel side L + f - 1,
                                     // camera window side (Le - 1) / f + 1 (f = 1: L, L)
    const double* Ke64;              // Le*Le effective kernel K (x) box_f (f = 1: the PSF itself)
    const float* Ke32;
    int sample_every, n_samples;     // kept objects: every sample_every-th sweep past burn-in, n_samples slots
    const double* adapt_fac;         // [burn_in][2] proposal-scale factors after accept / reject, or null
};

// One chain (an instance of a problem with its own state and random stream).
struct Chain {
    int img, chain;
    void* rho;                       // Ho*Wo, T
    void* mu;                        // H*mu_pitch, T
    void* spec;                      // spec_len complex T
    float4* cum;                     // H*mu_pitch photon-posterior cumulants c1..c4 (float chains) or null
    float2* cum2;                    // H*mu_pitch cumulants c5, c6
    double* rho_sum;                 // Ho*Wo
    double* rho_sq;                  // Ho*Wo or null
    double* trace_part;              // [slot][patch] accepted dL + dP
    unsigned long long* acc_count;   // [sweep - 1]
    uint8_t* acc_log;                // [sweep - 1][Ho*Wo] or null
    int* prog;                       // per tile, kProgStride ints apart: progress word (steps published in
                                     // this launch, change marks)
    double* trace;                   // [sweep 0..max_sweeps]
    int tpi, tpj, nti, ntj;          // tile shape (patches) and tile grid
    int cta_base;                    // first block of this chain in the sweep grid
    int* tdev;                       // sweeps this chain has completed (device counter, advanced by k_trace)
    int n_sweeps;                    // sweeps of this chain in the launch (0: the launch's n_sweeps)
    void* samples;                   // [n_samples][Ho*Wo] T kept objects, or null
    void* steps;                     // [Ho*Wo] T per-pixel proposal scales (adapting problems), or null
    void* phi;                       // [H*mu_pitch] T photon counts (augmented sampler), or null
    const void* tmap;                // float marginal camera-grid chains: three 128-byte TMA tensor maps
                                     // (mu, cumulants c1..c4, c5..c6) for window staging, or null
};

// Window pixels per thread fetched in one batch by the sweep kernel, and by
// its lean form (which has a 64-register budget: 4 resident 256-thread
// blocks per SM instead of 3)
constexpr int kMaxPx = 4;
constexpr int kLeanPx = 2;
constexpr int kLeanMinCells = 256;   // the lean form by default for PSF windows larger than this

struct SweepArgs {
    const Image* imgs;
    const Chain* chains;
    int n_chains;
    int n_sweeps;                    // sweeps in this launch (chains may take fewer)
    int aug;                         // photon-count augmented sampler (every chain of the launch)
    int fine;                        // object lattices finer than the camera (every chain of the launch)
    int* err;
    int resident;                    // 1: tile state (data, spectra, rho) held in shared memory
    unsigned long long wait_ns;      // limit of each neighbour wait
    int silent_block;                // test knob: this block never publishes progress (-1: none)
    int solo;                        // every block updates one patch with one team (tiles of one patch,
                                     // block = team): the float resident camera-grid kernel (marginal and
                                     // augmented) has a form compiled for this plan
    int stage;                       // 1: window staging -- each update's expected-image and cumulant window
                                     // (and, streamed, its patch spectrum) copied to shared memory by the TMA
                                     // engine, the next round's while the current one computes; 0: none
    int lean;                        // 1: the lean float form (fewer window cells in flight per thread, a
                                     // 64-register budget, more resident warps); same results
};

// Window staging (float marginal sampler on the camera grid).  The window of
// the update of object pixel (i, j) is the camera box rows i-2R..i, columns
// j-2R..j; it is copied as a box of kStageW(L) columns starting at column
// x0 = (j - 2R) rounded down to a multiple of 4 (a TMA copy must start on a
// 16-byte boundary), L rows, from three tensors: mu (float), the cumulants
// c1..c4 (float4 per pixel, 4 floats) and c5, c6 (float2, 2 floats).  Cells
// outside the frame are filled with zeros (mu = 0 never occurs inside the
// frame).  A box side is at most 256 elements, so staging needs
// 4 kStageW(L) <= 256, i.e. L <= 61.
constexpr int kStageMaxL = 61;
__host__ __device__ inline int stage_w(int L) { return (L + 6) & ~3; }   // round_up_4(L + 3)
__host__ __device__ inline size_t al128(size_t x) { return (x + 127) & ~(size_t)127; }
struct StagePlan {
    size_t mu, cum, cum2, spec, per_buf, bar;   // offsets within one buffer; bytes per buffer
    uint32_t tx_win, tx_spec;                   // bytes each copy set delivers
};
// the window, and the spectrum when the tile state is not resident
__host__ __device__ inline StagePlan stage_plan(int L, int max_nhalf, int mode, int resident)
{
    StagePlan p;
    const size_t cells = mode == 1 ? (size_t)stage_w(L) * L : 0;
    size_t o = 0;
    p.mu = o; o += al128(4 * cells);
    p.cum = o; o += al128(16 * cells);
    p.cum2 = o; o += al128(8 * cells);
    p.spec = o;
    // the half spectrum, rounded up to an even number of complex floats (16 bytes)
    const bool spec = mode == 1 && !resident;
    const size_t spec_bytes = spec ? (size_t)((max_nhalf + 1) & ~1) * 8 : 0;
    o += al128(spec_bytes);
    p.per_buf = o;
    p.tx_win = (uint32_t)(28 * cells);
    p.tx_spec = (uint32_t)spec_bytes;
    p.bar = 0;
    return p;
}

// Threads that cooperate on one pixel update, sized by the PSF side: one warp
// per 100 window pixels, 1..8 warps (at most 4 window pixels per thread up to
// L = 32).  The team of a problem is fixed by the problem alone (see
// problem_team), so its arithmetic and reduction order never depend on the
// launch plan or on the other problems of a batch.
__host__ __device__ inline int team_threads(int L)
{
    int w = (L * L + 99) / 100;
    w = w < 1 ? 1 : (w > 8 ? 8 : w);
    return 32 * w;
}

// Team of a problem: the requested warps; else, when the problem alone has
// many independent updates per class step (chains x patches >= 2048:
// throughput comes from many updates in flight), a small team -- in float,
// 1 warp up to 128 window pixels, 2 up to 600, 4 beyond (measured best on
// the 64-frame batch and the 2048 x 2048 frame: larger windows are
// latency-bound on one warp); in double 1 warp (the double sweep is bound by
// its arithmetic); else team_threads(L) (few updates per step: latency comes
// from the length of each update).
__host__ __device__ inline int problem_team(int L, int n_chains, int n_patches, int team_warps, bool fp32)
{
    if (team_warps > 0) return 32 * (team_warps > 8 ? 8 : team_warps);
    if ((long long)n_chains * n_patches >= 2048) return !fp32 || L * L <= 128 ? 32 : L * L <= 600 ? 64 : 128;
    return team_threads(L);
}

// Dynamic shared memory of one sweep block: fixed tables, reduction scratch
// and (resident plans) the tile's data constants with PSF halo, its patch
// spectra and its object values.
__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }
struct SmemPlan {
    size_t red, K, tw, ekl, ewa, em, prop, spec, rho, dat, stage, stage_bar, total;
};

// Proposal ring of a sweep block: per update team, the draws (s_m z, log u,
// rho', delta) of its next kPropRing updates, made ahead by one warp.
constexpr int kPropRing = 32;

// Progress words are kProgStride ints apart (one 128-byte line per tile), so
// that the neighbours' polls and the tile's publishes of different tiles do
// not meet on the same L2 lines.
constexpr int kProgStride = 32;
__host__ __device__ inline SmemPlan smem_plan(int L, int f, int S, int n_tw, int n_ent, int max_nhalf, int tpi,
                                              int tpj, int resident, int tsize, int teams, int stage = 0,
                                              bool lean = false)
{
    SmemPlan p;
    size_t o = 0;
    const int Le = L + f - 1, Lc = (Le - 1) / f + 1;
    // partial sums [prior, likelihood][8 sub-teams][8 warps][4]; two sets in
    // two-team blocks of the lean form, whose later rounds alternate between them
    p.red = o; o += al16((size_t)(lean && teams == 2 && !stage ? 2 : 1) * 2 * 8 * 8 * 4 * tsize);
    p.K = o; o += al16((size_t)Le * Le * tsize);
    p.tw = o; o += al16((size_t)2 * n_tw * tsize);
    p.ekl = o; o += al16((size_t)4 * n_ent);
    p.ewa = o; o += al16((size_t)n_ent * tsize);
    p.em = o; o += al16((size_t)n_ent * tsize);
    p.prop = o; o += al16((size_t)teams * kPropRing * 4 * tsize);
    if (resident) {
        const int R = L / 2;
        // camera rows / columns seen by the tile's windows
        const int ch = f == 1 ? tpi * S + 2 * R : (tpi * S + f - 1) / f + Lc;
        const int cw = f == 1 ? tpj * S + 2 * R : (tpj * S + f - 1) / f + Lc;
        p.spec = o; o += al16((size_t)tpi * tpj * max_nhalf * 2 * tsize);
        p.rho = o; o += al16((size_t)tpi * tpj * S * S * tsize);
        p.dat = o; o += al16((size_t)ch * cw * 4 * tsize);
    } else {
        p.spec = p.rho = p.dat = o;
    }
    p.stage = p.stage_bar = o;
    if (stage) {
        // per update team: two staging buffers (the current round's and the next
        // one's) and their two completion barriers
        o = al128(o);
        p.stage = o;
        o += (size_t)teams * 2 * stage_plan(L, max_nhalf, stage, resident).per_buf;
        p.stage_bar = o;
        o += al16((size_t)teams * 2 * 8);
    }
    p.total = o;
    return p;
}

// host launchers (defined in the .cu files)
void launch_setup(const Image& im, const Image* d_im, const float* w, const float* g,
                  const float* o, const float* v, double gs, double os, double vs,
                  const double* psf_raw, double* b0_out, double* scratch, cudaStream_t st,
                  int64_t* launches);
template <typename T>
void launch_init_rho(const Image& im, const Chain& ch, const double* b0, cudaStream_t st,
                     int64_t* launches);
template <typename T>
// out_logpost receives the log posterior at out_logpost[*out_index] (index 0
// when out_index is null)
// (with write_state on an augmented chain, the total is the log of the joint
// density p(w, phi, rho) at the chain's photon counts)
void launch_refresh(const Image& im, const Chain& ch, double* scratch, int write_state,
                    double* out_logpost, const int* out_index, int* err, cudaStream_t st, int64_t* launches);
// photon counts of every camera pixel drawn from p(phi | w, mu) with the
// uniforms of sweep t (the augmented sampler's initial draw)
template <typename T>
void launch_sample_phi(const Image& im, const Chain& ch, int t, int* err, cudaStream_t st, int64_t* launches);
template <typename T>
cudaError_t launch_sweep(const SweepArgs& a, int grid, int threads, size_t smem, cudaStream_t st);
template <typename T>
int sweep_blocks_per_sm(int threads, size_t smem, bool aug, bool fine, int stg, bool solo, bool lean);
// zero every chain's progress words and trace partials
void launch_reset(const Image* d_imgs, const Chain* d_chains, int n_chains, int n_slots, cudaStream_t st,
                  int64_t* launches);
void launch_trace(const Image* d_imgs, const Chain* d_chains, int n_chains, int n_sweeps,
                  cudaStream_t st, int64_t* launches);
template <typename T>
void launch_delta(const Image* d_im, const Chain* d_ch, int64_t m, double rho_new, double* out3, int team,
                  cudaStream_t st, int64_t* launches);
template <typename T>
void launch_convert(const void* src, double* dst, int64_t n, int rows, int cols, int src_pitch,
                    cudaStream_t st, int64_t* launches);
template <typename T>
void launch_set_rho(const double* src, void* dst, int64_t n, cudaStream_t st, int64_t* launches);
template <typename T>
void launch_fill(void* dst, int64_t n, double value, cudaStream_t st, int64_t* launches);
// sets every chain's sweep counter to value
void launch_set_counters(const Chain* d_chains, int n_chains, int value, cudaStream_t st, int64_t* launches);
// sets the thread-local message that bdecon_last_error(NULL) returns
void set_host_error(const char* msg);
// pooled map of the chains' running sums: kind 0 mean, 1 variance, 2 standard
// deviation, 3 coefficient of variation (1-3 need the sums of squares sq)
void launch_mean(const double* sum, int n_chains_img, int64_t chain_stride_elems, int Ho, int Wo,
                 int crop_r, int out_h, int out_w, double inv_n, double* out, const double* sq,
                 int kind, cudaStream_t st, int64_t* launches);
constexpr int kMaxQuantiles = 64;
constexpr int kMaxQuantileValues = 8192;
// quantiles q[0..nq) of the kept objects (slots [first, first + count) of
// every chain; chain c's store at samples + c * chain_stride elements) for
// the object pixels pix0 .. pix0 + npix - 1 of the (cropped) output grid;
// out[k * npix + i] for quantile k of pixel pix0 + i
template <typename T>
cudaError_t launch_quantiles(const void* samples, int64_t chain_stride, int n_chains, int first, int count,
                             int64_t obj_pixels, int Wo, int crop_r, int out_w, int64_t pix0, int64_t npix,
                             const double* q, int nq, double* out, cudaStream_t st, int64_t* launches);

}  // namespace bd
