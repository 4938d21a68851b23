// bdecon_api.cu -- host side of the libbdecon C ABI (see include/bdecon.h):
// argument validation, the device arena, the launch plan of the persistent
// sweep kernel, and the sweep / refresh / trace schedule.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "bdecon.h"
#include "bd_internal.h"

using namespace bd;

namespace {

thread_local std::string g_err;

}  // namespace

void bd::set_host_error(const char* msg) { g_err = msg; }

namespace {

struct ProbHost {
    bdecon_problem p;           // copy (host pointers not retained)
    int H, W, L, R, S, Ho, Wo, npi, npj, n_patches, pitch;
    int f = 1, Le = 0, Lc = 0;  // lattice cells per camera pixel side, effective kernel side, window side
    int tpi = 1, tpj = 1;       // tile shape in patches
    bool user_plan = false;
    int64_t n_sum = 0;          // sweeps averaged so far
    Shape shape[kMaxShapes];
    std::vector<int> ent_kl;
    std::vector<int64_t> patch_off;
    int64_t spec_len = 0;
    int n_tw = 0;               // complex twiddle entries
    int max_nhalf = 0;
    // arena offsets (bytes)
    size_t o_Ke64 = 0, o_Ke32 = 0;
    size_t o_K64, o_K32, o_dat64, o_dat32, o_ekl, o_wa64, o_m64, o_wa32, o_m32, o_tw64, o_tw32, o_poff;
    size_t o_sum, o_sq, o_scr, o_samp, o_adapt;
    int samp_first = 0;         // first valid kept-object slot (after a resume)
    bool stage_ok = false;      // its chains carry TMA tensor maps for window staging
    bool many = false;          // many independent updates per class step (its team chosen for throughput)
    size_t scr_doubles;
    int chain0;
};

// Problems with the same PSF side, stride and update team share a launch:
// they have the same number of class steps per sweep and the same block.
struct Group {
    std::vector<int> probs;
    int L = 0, S = 0, team = 32;
    int threads = 32, warps = 1;
    bool user_warps = false;
    int grid = 0;
    size_t smem = 0;
    int resident = 1;
    bool streamed = false;             // plan with tile state in global memory even if it fits in shared
    bool aug = false;                  // photon-count augmented problems (their own kernel form)
    bool fine = false;                 // object lattices finer than the camera (their own kernel form)
    bool solo = false;                 // every block: one patch, one team (a kernel form of its own)
    int stage = 0;                     // window staging by the TMA engine (a kernel form): 1 on, 0 off
    bool no_stage = true;              // window staging not allowed in this group's plan
    bool many = false;                 // every problem has many updates per class step: two teams per block
    bool user_stage = false;           // no_stage set by the autotuner, not by the handle's setting
    int lean_mode = -1;                // lean kernel form: -1 automatic, 0 off, 1 on where eligible
    int user_lean = -2;                // lean_mode set by the autotuner (-2: not set; the handle's setting)
    bool lean = false;                 // the plan runs the lean form
    int chain_off = 0, n_chains = 0;   // slice of the group-ordered chain table
};

struct ChainHost {
    size_t o_rho, o_mu, o_spec, o_cum, o_cum2, o_tpart, o_acc, o_log, o_prog, o_trace, o_tdev, o_steps, o_phi;
    size_t o_tmap = 0;
};

}  // namespace

struct bdecon_handle {
    std::vector<ProbHost> probs;
    std::vector<ChainHost> chh;
    std::vector<Image> imgs;
    std::vector<Chain> chains;
    int precision = 1;
    int max_sweeps = 4096;
    int64_t sweeps = 0;
    std::vector<Group> groups;
    bool one_launch = false;            // all problems in one launch instead of one per (L, S, team)
    int staging = 0;                    // window staging by the TMA engine in eligible groups (1) or not (0)
    int lean = -1;                      // lean kernel form: -1 automatic, 0 off, 1 on where eligible
    std::vector<int> prob_group;        // problem -> group
    std::vector<Chain> gch;             // host copy of the group-ordered chain table
    size_t o_gchains = 0;
    Chain* d_gchains = nullptr;          // chain descriptors in group order
    bool failed = false;
    int sms = 0;
    cudaStream_t st = nullptr;
    char* arena = nullptr;
    size_t arena_bytes = 0;
    bool own_arena = false;
    size_t o_imgs = 0, o_chains = 0, o_err = 0, o_out = 0, o_scr = 0, o_up = 0;
    size_t up_bytes = 0;
    Image* d_imgs = nullptr;
    Chain* d_chains = nullptr;
    int* d_err = nullptr;
    double* d_out = nullptr;        // small read-out buffer
    double* d_up = nullptr;         // staging buffer for set_state / results
    int64_t launches = 0;
    bool timing = false;
    int silent_block = -1;              // test knob (bdecon_set_fault)
    unsigned long long wait_ns = 4000000000ull;
    std::vector<cudaEvent_t> ev_pool;    // pairs (start, stop), reused
    size_t ev_used = 0;
    // CUDA-graph mode: the kernel sequence of one bdecon_sweep call, keyed by
    // its segment lengths and refreshes, captured once and replayed
    bool use_graph = false;
    struct GraphEntry {
        std::vector<int> sig;
        cudaGraphExec_t exec = nullptr;
        int64_t launches = 0;
    };
    std::vector<GraphEntry> graphs;
    cudaStream_t cap_st = nullptr;
    std::string err;
};

namespace {

bdecon_status fail(bdecon_handle* h, bdecon_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf; else g_err = buf;
    return s;
}

#define CK(h, call)                                                                         \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) return fail((h), BDECON_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Alloc {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        off = align_up(off, 256);
        size_t r = off;
        off += bytes;
        return r;
    }
};

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

bdecon_status validate(const bdecon_problem& p, int idx)
{
    if (p.H < 1 || p.W < 1 || p.H > 16384 || p.W > 16384)
        return fail(nullptr, BDECON_ERR_INVALID, "problem %d: frame size %dx%d out of range", idx, p.H, p.W);
    if (!p.image || !p.psf) return fail(nullptr, BDECON_ERR_INVALID, "problem %d: image and psf are required", idx);
    if (p.L < 1 || p.L > kMaxL || p.L % 2 == 0)
        return fail(nullptr, BDECON_ERR_INVALID, "problem %d: PSF side %d must be odd and <= %d", idx, p.L, kMaxL);
    if (p.subpixel < 0 || p.subpixel > 8) return fail(nullptr, BDECON_ERR_INVALID, "problem %d: subpixel %d", idx, p.subpixel);
    const int f = p.subpixel > 1 ? p.subpixel : 1, Le = p.L + f - 1;
    const int S = p.stride ? p.stride : Le;
    if (S < Le || S > kMaxS)
        return fail(nullptr, BDECON_ERR_INVALID, "problem %d: stride %d must be in [L + subpixel - 1 = %d, %d]", idx, S,
                    Le, kMaxS);
    if (p.n_chains < 1 || p.n_chains > 4096) return fail(nullptr, BDECON_ERR_INVALID, "problem %d: n_chains %d", idx, p.n_chains);
    if (p.team_warps < 0 || p.team_warps > 8) return fail(nullptr, BDECON_ERR_INVALID, "problem %d: team_warps %d", idx, p.team_warps);
    if (!(p.adapt_target >= 0.0 && p.adapt_target < 1.0))
        return fail(nullptr, BDECON_ERR_INVALID, "problem %d: adapt_target must be in [0, 1)", idx);
    if (p.n_samples < 0 || p.sample_every < 0)
        return fail(nullptr, BDECON_ERR_INVALID, "problem %d: n_samples %d / sample_every %d must be >= 0", idx, p.n_samples,
                    p.sample_every);
    if (p.precision != BDECON_FP32 && p.precision != BDECON_FP64)
        return fail(nullptr, BDECON_ERR_INVALID, "problem %d: precision %d", idx, p.precision);
    if (p.burn_in < 0 || p.refresh_every < 0 || p.max_sweeps < 0)
        return fail(nullptr, BDECON_ERR_INVALID, "problem %d: negative burn_in/refresh_every/max_sweeps", idx);
    if (!(p.step >= 0.0) || !std::isfinite(p.step)) return fail(nullptr, BDECON_ERR_INVALID, "problem %d: step", idx);
    double s = 0.0;
    for (int k = 0; k < p.L * p.L; ++k) {
        if (!std::isfinite(p.psf[k]) || p.psf[k] < 0.0)
            return fail(nullptr, BDECON_ERR_INVALID, "problem %d: PSF entry %d is negative or not finite", idx, k);
        s += p.psf[k];
    }
    if (!(s > 0.0)) return fail(nullptr, BDECON_ERR_INVALID, "problem %d: PSF sums to zero", idx);
    const int64_t n = (int64_t)p.H * p.W;
    for (int64_t k = 0; k < n; ++k)
        if (!std::isfinite(p.image[k])) return fail(nullptr, BDECON_ERR_INVALID, "problem %d: image[%lld] not finite", idx, (long long)k);
    if (p.gain_map) {
        for (int64_t k = 0; k < n; ++k)
            if (!finite_pos(p.gain_map[k])) return fail(nullptr, BDECON_ERR_INVALID, "problem %d: gain_map[%lld] must be > 0", idx, (long long)k);
    } else if (!finite_pos(p.gain)) return fail(nullptr, BDECON_ERR_INVALID, "problem %d: gain must be > 0", idx);
    if (p.var_map) {
        for (int64_t k = 0; k < n; ++k)
            if (!finite_pos(p.var_map[k])) return fail(nullptr, BDECON_ERR_INVALID, "problem %d: var_map[%lld] must be > 0", idx, (long long)k);
    } else if (!finite_pos(p.read_var)) return fail(nullptr, BDECON_ERR_INVALID, "problem %d: read_var must be > 0", idx);
    if (p.offset_map) {
        for (int64_t k = 0; k < n; ++k)
            if (!std::isfinite(p.offset_map[k])) return fail(nullptr, BDECON_ERR_INVALID, "problem %d: offset_map not finite", idx);
    } else if (!std::isfinite(p.offset)) return fail(nullptr, BDECON_ERR_INVALID, "problem %d: offset not finite", idx);
    return BDECON_OK;
}

// canonical half of the ph x pw frequencies: (k, l) kept iff it is not larger
// (lexicographically) than its conjugate partner ((-k) mod ph, (-l) mod pw)
void half_entries(int ph, int pw, std::vector<int>& out)
{
    for (int k = 0; k < ph; ++k)
        for (int l = 0; l < pw; ++l) {
            const int kc = (ph - k) % ph, lc = (pw - l) % pw;
            if (k < kc || (k == kc && l <= lc)) out.push_back((k << 16) | l);
        }
}

void describe(ProbHost& ph)
{
    const bdecon_problem& p = ph.p;
    ph.H = p.H; ph.W = p.W; ph.L = p.L; ph.R = p.L / 2;
    ph.f = p.subpixel > 1 ? p.subpixel : 1;
    ph.Le = p.L + ph.f - 1;
    ph.Lc = (ph.Le - 1) / ph.f + 1;
    ph.S = p.stride ? p.stride : ph.Le;
    ph.Ho = ph.f * p.H + 2 * ph.R; ph.Wo = ph.f * p.W + 2 * ph.R;
    ph.npi = (ph.Ho + ph.S - 1) / ph.S; ph.npj = (ph.Wo + ph.S - 1) / ph.S;
    ph.n_patches = ph.npi * ph.npj;
    ph.pitch = (int)align_up((size_t)p.W, 4);
    const int rh = ph.Ho - (ph.npi - 1) * ph.S, rw = ph.Wo - (ph.npj - 1) * ph.S;   // last patch sides
    int twoff = 0;
    ph.ent_kl.clear();
    ph.max_nhalf = 0;
    for (int s = 0; s < kMaxShapes; ++s) {
        Shape& sh = ph.shape[s];
        const bool pr = (s & 2) != 0, pc = (s & 1) != 0;
        // a shape exists if some patch has it
        const bool exists = (!pr || rh < ph.S) && (!pc || rw < ph.S);
        std::memset(&sh, 0, sizeof sh);
        if (!exists) continue;
        sh.ph = pr ? rh : ph.S;
        sh.pw = pc ? rw : ph.S;
        sh.K = sh.ph * sh.pw;
        sh.ent_off = (int)ph.ent_kl.size();
        half_entries(sh.ph, sh.pw, ph.ent_kl);
        sh.nhalf = (int)ph.ent_kl.size() - sh.ent_off;
        ph.max_nhalf = std::max(ph.max_nhalf, sh.nhalf);
        sh.twh_off = twoff; twoff += sh.ph;
        sh.tww_off = twoff; twoff += sh.pw;
        sh.inv_ph = 1.0f / (float)sh.ph;
        sh.inv_pw = 1.0f / (float)sh.pw;
    }
    ph.n_tw = twoff;
    ph.patch_off.resize(ph.n_patches);
    int64_t off = 0;
    for (int pi = 0; pi < ph.npi; ++pi)
        for (int pj = 0; pj < ph.npj; ++pj) {
            const int s = (((pi + 1) * ph.S > ph.Ho) ? 2 : 0) | (((pj + 1) * ph.S > ph.Wo) ? 1 : 0);
            ph.patch_off[pi * ph.npj + pj] = off;
            // even offsets: every patch's half spectrum starts 16-byte aligned in
            // float (the staged plans copy it with one bulk copy)
            off += (ph.shape[s].nhalf + 1) & ~1;
        }
    ph.spec_len = off;
}

// Blocks per SM of the sweep kernel's forms for this launch shape, memoized:
// the planner asks at every tile-growth step, and the answer depends only on
// the device, the precision, the block size, the shared memory and the form.
int occupancy(int prec, int threads, size_t smem, bool aug, bool fine, int stg, bool solo = false, bool lean = false)
{
    static std::mutex mu;
    static std::map<std::vector<long long>, int> memo;
    int dev = 0;
    cudaGetDevice(&dev);
    const std::vector<long long> key = {dev, prec, threads, (long long)smem, aug ? 1 : 0, fine ? 1 : 0, stg, solo ? 1 : 0,
                                        lean ? 1 : 0};
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = memo.find(key);
        if (it != memo.end()) return it->second;
    }
    const int n = prec == BDECON_FP32 ? sweep_blocks_per_sm<float>(threads, smem, aug, fine, stg, solo, lean)
                                      : sweep_blocks_per_sm<double>(threads, smem, aug, fine, stg, solo, lean);
    if (n > 0) {
        std::lock_guard<std::mutex> lock(mu);
        memo[key] = n;
    }
    return n;
}

constexpr size_t kMaxSmem = 227 * 1024;

// One problem's entry in a launch plan: the problem, its update team, its
// tile shape, and its chains' descriptors in the launch's chain table.
struct PlanItem {
    const ProbHost* ph = nullptr;
    int team = 32;
    int tpi = 1, tpj = 1;
    bool user = false;
    std::vector<Chain*> chains;
};

int item_blocks(const PlanItem& it)
{
    return (int)it.chains.size() * ((it.ph->npi + it.tpi - 1) / it.tpi) * ((it.ph->npj + it.tpj - 1) / it.tpj);
}

size_t items_smem(const std::vector<PlanItem*>& items, int resident, int ts, int threads, int stage,
                  bool lean = false)
{
    size_t mx = 0;
    for (const PlanItem* it : items) {
        const ProbHost& ph = *it->ph;
        const int teams = std::max(1, threads / it->team);   // update teams per block
        const SmemPlan sp = smem_plan(ph.L, ph.f, ph.S, ph.n_tw, (int)ph.ent_kl.size(), ph.max_nhalf, it->tpi,
                                      it->tpj, resident, ts, teams, stage, lean);
        mx = std::max(mx, sp.total);
    }
    return mx;
}

// Grow the tile of the problem whose tiles are smallest (ties: the one with
// the most blocks); false if none can grow.  A launch lasts as long as its
// slowest chain, and a block takes one round per patch of its tile at every
// class step, so the launch is fastest when every problem's tiles hold about
// the same number of patches; growing the problem with the most blocks
// instead gives the largest frames of a batch the largest tiles.
bool grow_items(std::vector<PlanItem*>& items)
{
    PlanItem* worst = nullptr;
    int wa = 1 << 30, wb = -1;
    for (PlanItem* it : items) {
        if (it->user || (it->tpi >= it->ph->npi && it->tpj >= it->ph->npj)) continue;
        const int area = std::min(it->tpi, it->ph->npi) * std::min(it->tpj, it->ph->npj);
        const int b = item_blocks(*it);
        if (area < wa || (area == wa && b > wb)) {
            wa = area;
            wb = b;
            worst = it;
        }
    }
    if (!worst) return false;
    if ((worst->tpj <= worst->tpi && worst->tpj < worst->ph->npj) || worst->tpi >= worst->ph->npi) ++worst->tpj;
    else ++worst->tpi;
    return true;
}

// Launch plan of one group: block = the group's update team (or the user's
// warps); tiles grow from one patch until every block of every chain of the
// group is co-resident.  Resident plans (tile state in shared memory) are
// preferred; if none fits, tile state is streamed from global memory.
bool plan_items(int precision, int sms, std::vector<PlanItem*>& items, Group& g, std::string& err)
{
    int team = 32;
    for (const PlanItem* it : items) team = std::max(team, it->team);
    // default block: one update team; two when every problem has many updates
    // per class step (measured: the autotuner's usual choice for such groups)
    const int dflt = g.many && 2 * team <= 256 ? 2 * team : team;
    g.threads = g.user_warps ? std::max(32 * g.warps, team) : dflt;
    g.warps = g.threads / 32;
    const int ts = precision == BDECON_FP32 ? 4 : 8;
    // window staging: float marginal camera-grid problems whose chains carry
    // tensor maps, when the handle (or the autotuner) asks for it; a plan in
    // which every block updates one patch with one team keeps the one-team
    // form instead (its windows are read once per step from L2 by many blocks
    // at once, and it needs no buffers)
    bool stage_ok = precision == BDECON_FP32 && !g.aug && !g.fine && !g.no_stage;
    // lean form (unstaged float marginal camera-grid plans): automatically
    // for windows of more than kLeanMinCells cells (measured on the 64-frame
    // batch: faster from PSF side 17 up, slower at 9 and 13, where its extra
    // window batches cost more than its extra resident warps give)
    bool want_lean = precision == BDECON_FP32 && !g.aug && !g.fine && g.lean_mode != 0;
    if (want_lean && g.lean_mode < 0)
        for (const PlanItem* it : items) want_lean = want_lean && it->ph->L * it->ph->L > kLeanMinCells;
    for (const PlanItem* it : items) stage_ok = stage_ok && it->ph->stage_ok;
    bool done = false;
    for (int attempt = stage_ok ? 0 : 1; attempt < 2 && !done; ++attempt) {
        for (int resident = g.streamed ? 0 : 1; resident >= 0 && !done; --resident) {
            const int stage = attempt == 0 ? 1 : 0;
            for (PlanItem* it : items)
                if (!it->user) it->tpi = it->tpj = 1;
            for (;;) {
                const size_t smem = items_smem(items, resident, ts, g.threads, stage, want_lean && stage == 0);
                int tot = 0;
                for (const PlanItem* it : items) tot += item_blocks(*it);
                if (smem <= kMaxSmem) {
                    const int bps = occupancy(precision, g.threads, smem, g.aug, g.fine, stage, false,
                                              want_lean && stage == 0);
                    if (bps > 0 && tot <= bps * sms) {
                        g.smem = smem;
                        g.resident = resident;
                        g.stage = stage;
                        done = true;
                        break;
                    }
                } else if (resident) {
                    break;   // tiles only grow: resident state will not fit
                }
                if (!grow_items(items)) break;
            }
        }
        if (done && attempt == 0) {
            // a one-patch one-team plan without staging runs the one-team form
            bool solo_ok = true;
            std::vector<std::pair<int, int>> keep;
            for (PlanItem* it : items) keep.push_back({it->tpi, it->tpj});
            for (PlanItem* it : items) {
                if (!it->user) it->tpi = it->tpj = 1;
                solo_ok = solo_ok && it->tpi == 1 && it->tpj == 1 && g.threads == it->team;
            }
            if (solo_ok) {
                const size_t smem = items_smem(items, 1, ts, g.threads, 0);
                int tot = 0;
                for (const PlanItem* it : items) tot += item_blocks(*it);
                const int bps = smem <= kMaxSmem ? occupancy(precision, g.threads, smem, g.aug, g.fine, 0, true) : 0;
                if (bps > 0 && tot <= bps * sms) {
                    g.smem = smem;
                    g.resident = 1;
                    g.stage = 0;
                    break;
                }
            }
            for (size_t k = 0; k < items.size(); ++k) {
                items[k]->tpi = keep[k].first;
                items[k]->tpj = keep[k].second;
            }
        }
    }
    if (!done) {
        int tot = 0;
        for (const PlanItem* it : items) tot += item_blocks(*it);
        char buf[160];
        snprintf(buf, sizeof buf, "no launch plan: %d blocks of %d threads cannot all be co-resident", tot, g.threads);
        err = buf;
        return false;
    }
    g.solo = g.stage == 0;
    for (const PlanItem* it : items) g.solo = g.solo && it->tpi == 1 && it->tpj == 1 && g.threads == it->team;
    if (g.solo) {
        // a one-patch one-team plan found above was sized for the other forms:
        // it runs the one-team form only if that form's blocks are co-resident too
        int tot = 0;
        for (const PlanItem* it : items) tot += item_blocks(*it);
        const int bps = occupancy(precision, g.threads, g.smem, g.aug, g.fine, 0, true);
        if (!(bps > 0 && tot <= bps * sms)) g.solo = false;
    }
    g.lean = want_lean && g.stage == 0 && !g.solo;
    int base = 0;
    for (PlanItem* it : items) {
        const int nti = (it->ph->npi + it->tpi - 1) / it->tpi, ntj = (it->ph->npj + it->tpj - 1) / it->tpj;
        for (Chain* ch : it->chains) {
            ch->tpi = it->tpi; ch->tpj = it->tpj; ch->nti = nti; ch->ntj = ntj;
            ch->cta_base = base;
            base += nti * ntj;
        }
    }
    g.grid = base;
    return true;
}

void drop_graphs(bdecon_handle* h)
{
    for (auto& g : h->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
}

// The handle's own plan: one group per (L, S, team) of its problems.
bdecon_status make_plan(bdecon_handle* h)
{
    drop_graphs(h);   // captured launches carry the old grid and tables
    for (auto& g : h->groups) {
        if (!g.user_stage) g.no_stage = h->staging == 0;
        g.lean_mode = g.user_lean != -2 ? g.user_lean : h->lean;
        std::vector<PlanItem> items(g.probs.size());
        std::vector<PlanItem*> ptrs;
        for (size_t k = 0; k < g.probs.size(); ++k) {
            ProbHost& ph = h->probs[g.probs[k]];
            PlanItem& it = items[k];
            it.ph = &ph;
            it.team = h->imgs[g.probs[k]].team;
            it.tpi = ph.tpi;
            it.tpj = ph.tpj;
            it.user = ph.user_plan;
            for (int c = 0; c < ph.p.n_chains; ++c) it.chains.push_back(&h->chains[ph.chain0 + c]);
            ptrs.push_back(&it);
        }
        std::string err;
        if (!plan_items(h->precision, h->sms, ptrs, g, err)) return fail(h, BDECON_ERR_INVALID, "%s", err.c_str());
        for (size_t k = 0; k < g.probs.size(); ++k) {
            h->probs[g.probs[k]].tpi = items[k].tpi;
            h->probs[g.probs[k]].tpj = items[k].tpj;
        }
    }
    h->gch.clear();
    for (auto& g : h->groups) {
        g.chain_off = (int)h->gch.size();
        for (int k : g.probs) {
            const ProbHost& ph = h->probs[k];
            for (int c = 0; c < ph.p.n_chains; ++c) h->gch.push_back(h->chains[ph.chain0 + c]);
        }
        g.n_chains = (int)h->gch.size() - g.chain_off;
    }
    CK(h, cudaMemcpyAsync(h->d_chains, h->chains.data(), sizeof(Chain) * h->chains.size(), cudaMemcpyHostToDevice, h->st));
    CK(h, cudaMemcpyAsync(h->d_gchains, h->gch.data(), sizeof(Chain) * h->gch.size(), cudaMemcpyHostToDevice, h->st));
    return BDECON_OK;
}

// Launch groups: one per (L, S, team), or a single group when one_launch is
// set (the kernel reads each block's problem from its chain; the block size
// is then the largest team and the shared memory the largest tile plan).
void form_groups(bdecon_handle* h)
{
    const int n = (int)h->probs.size();
    h->groups.clear();
    h->prob_group.assign(n, -1);
    for (int k = 0; k < n; ++k) {
        int gi = -1;
        const bool aug = (h->probs[k].p.flags & BDECON_FLAG_AUGMENTED) != 0;
        const bool fine = h->probs[k].f > 1;
        for (size_t q = 0; q < h->groups.size() && gi < 0; ++q)
            if (h->groups[q].aug == aug && h->groups[q].fine == fine &&
                (h->one_launch || (h->groups[q].L == h->probs[k].L && h->groups[q].S == h->probs[k].S &&
                                   h->groups[q].team == h->imgs[k].team)))
                gi = (int)q;
        if (gi < 0) {
            Group g;
            g.L = h->probs[k].L;
            g.S = h->probs[k].S;
            g.team = h->imgs[k].team;
            g.aug = aug;
            g.fine = fine;
            h->groups.push_back(g);
            gi = (int)h->groups.size() - 1;
        }
        h->groups[gi].probs.push_back(k);
        h->prob_group[k] = gi;
    }
    for (auto& g : h->groups) {
        g.many = true;
        for (int k : g.probs) g.many = g.many && h->probs[k].many;
    }
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (no link-time dependency on the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    });
    return fn;
}

// The window-staging tensor maps of one float chain: mu (H x W floats, row
// pitch mu_pitch), the cumulants c1..c4 (H x 4W floats) and c5, c6 (H x 2W
// floats); boxes of stage_w(L) pixels by L rows, zeros outside the frame.
bool encode_stage_maps(const ProbHost& ph, const Chain& ch, CUtensorMap out[3])
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint32_t BW = (cuuint32_t)stage_w(ph.L), L = (cuuint32_t)ph.L;
    const cuuint32_t es[2] = {1, 1};
    void* base[3] = {ch.mu, ch.cum, ch.cum2};
    const int per[3] = {1, 4, 2};   // floats per pixel
    for (int k = 0; k < 3; ++k) {
        const cuuint64_t dims[2] = {(cuuint64_t)per[k] * ph.W, (cuuint64_t)ph.H};
        const cuuint64_t strides[1] = {(cuuint64_t)per[k] * 4 * ph.pitch};
        const cuuint32_t box[2] = {per[k] * BW, L};
        if (enc(&out[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base[k], dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}

size_t layout(bdecon_handle* h, std::vector<ProbHost>& probs, std::vector<ChainHost>& chh, int prec, int max_sweeps)
{
    Alloc A;
    const size_t ts = prec == BDECON_FP32 ? 4 : 8;
    size_t up = 0;
    size_t scr_max = 0;
    chh.clear();
    for (auto& ph : probs) {
        const size_t npix = (size_t)ph.H * ph.W, nobj = (size_t)ph.Ho * ph.Wo, nh = ph.ent_kl.size();
        ph.o_K64 = A.take(8 * ph.L * ph.L);
        ph.o_K32 = A.take(4 * ph.L * ph.L);
        if (ph.f > 1) {
            ph.o_Ke64 = A.take(8 * (size_t)ph.Le * ph.Le);
            ph.o_Ke32 = A.take(4 * (size_t)ph.Le * ph.Le);
        }
        ph.o_dat64 = A.take(32 * npix);
        ph.o_dat32 = A.take(16 * npix);
        ph.o_ekl = A.take(4 * nh);
        ph.o_wa64 = A.take(8 * nh);
        ph.o_m64 = A.take(8 * nh);
        ph.o_wa32 = A.take(4 * nh);
        ph.o_m32 = A.take(4 * nh);
        ph.o_tw64 = A.take(16 * ph.n_tw);
        ph.o_tw32 = A.take(8 * ph.n_tw);
        ph.o_poff = A.take(8 * ph.n_patches);
        ph.o_sum = A.take(8 * nobj * ph.p.n_chains);
        ph.o_sq = (ph.p.flags & BDECON_FLAG_SECOND_MOMENT) ? A.take(8 * nobj * ph.p.n_chains) : 0;
        ph.o_samp = ph.p.n_samples > 0 ? A.take(ts * nobj * (size_t)ph.p.n_samples * ph.p.n_chains) : 0;
        const bool adapt = ph.p.adapt_target > 0.0 && ph.p.burn_in > 0;
        ph.o_adapt = adapt ? A.take(16 * (size_t)ph.p.burn_in) : 0;
        const size_t nblk = (npix + kRedThreads - 1) / kRedThreads;
        ph.scr_doubles = std::max(nblk + (size_t)ph.n_patches + 8, nblk + 8 + 2 * (size_t)kMaxS * kMaxS) + 8;
        ph.o_scr = A.take(8 * ph.scr_doubles);
        scr_max = std::max(scr_max, ph.scr_doubles);
        up = std::max(up, std::max(16 * npix + 8 * (size_t)ph.L * ph.L, 8 * nobj));
        ph.chain0 = (int)chh.size();
        for (int c = 0; c < ph.p.n_chains; ++c) {
            ChainHost x;
            x.o_rho = A.take(ts * nobj);
            x.o_mu = A.take(ts * (size_t)ph.H * ph.pitch);
            x.o_spec = A.take(2 * ts * (size_t)ph.spec_len);
            const bool aug = (ph.p.flags & BDECON_FLAG_AUGMENTED) != 0;
            x.o_cum = prec == BDECON_FP32 && !aug ? A.take(16 * (size_t)ph.H * ph.pitch) : 0;
            x.o_cum2 = prec == BDECON_FP32 && !aug ? A.take(8 * (size_t)ph.H * ph.pitch) : 0;
            x.o_phi = aug ? A.take(ts * (size_t)ph.H * ph.pitch) : 0;
            x.o_tpart = A.take(8 * (size_t)kMaxSlots * ph.n_patches);
            x.o_acc = A.take(8 * (size_t)max_sweeps);
            x.o_log = (ph.p.flags & BDECON_FLAG_ACCEPT_LOG) ? A.take((size_t)max_sweeps * nobj) : 0;
            x.o_prog = A.take(4 * (size_t)ph.n_patches * kProgStride);
            x.o_trace = A.take(8 * ((size_t)max_sweeps + 1));
            x.o_tdev = A.take(4);
            x.o_steps = adapt ? A.take(ts * nobj) : 0;
            // window staging: three 128-byte TMA tensor maps (64-byte aligned)
            x.o_tmap = prec == BDECON_FP32 && !aug && ph.f == 1 && ph.L <= kStageMaxL ? A.take(3 * sizeof(CUtensorMap)) : 0;
            chh.push_back(x);
        }
    }
    h->o_imgs = A.take(sizeof(Image) * probs.size());
    h->o_chains = A.take(sizeof(Chain) * chh.size());
    h->o_gchains = A.take(sizeof(Chain) * chh.size());
    h->o_err = A.take(64);
    h->o_out = A.take(64);
    h->up_bytes = up;
    h->o_up = A.take(up);
    (void)scr_max;
    return align_up(A.off, 256);
}

// Double refresh of chain ci (mu, spectra, cumulant cache when write is set)
// and its log posterior into out[*idx] (out[0] when idx is null).
template <typename T>
bdecon_status refresh_chain(bdecon_handle* h, int ci, int write, double* out, const int* idx)
{
    const Chain& ch = h->chains[ci];
    const ProbHost& ph = h->probs[ch.img];
    launch_refresh<T>(h->imgs[ch.img], ch, (double*)(h->arena + ph.o_scr), write, out, idx, h->d_err, h->st,
                      &h->launches);
    CK(h, cudaGetLastError());
    return BDECON_OK;
}

bdecon_status refresh(bdecon_handle* h, int ci, int write, double* out, const int* idx = nullptr)
{
    return h->precision == BDECON_FP32 ? refresh_chain<float>(h, ci, write, out, idx)
                                       : refresh_chain<double>(h, ci, write, out, idx);
}

bdecon_status check_device(bdecon_handle* h)
{
    int e[10] = {};
    CK(h, cudaStreamSynchronize(h->st));
    CK(h, cudaMemcpy(e, h->d_err, sizeof e, cudaMemcpyDeviceToHost));
    if (e[0] & kErrTimeout) { h->failed = true; return fail(h, BDECON_ERR_TIMEOUT, "a sub-lattice wait timed out on the device"); }
    if (e[0] & kErrNumeric) { h->failed = true; return fail(h, BDECON_ERR_NUMERIC, "non-finite or non-positive expected image"); }
    if (e[0] & kErrRatio) {
        double d[2];
        std::memcpy(d, e + 4, sizeof d);
        h->failed = true;
        return fail(h, BDECON_ERR_NUMERIC,
                    "non-finite log acceptance ratio (first: chain %d, object pixel %d, sweep %d, dL %g, dP %g); "
                    "the update was rejected",
                    e[2], e[3], e[8], d[0], d[1]);
    }
    return BDECON_OK;
}

struct TuneChoice {
    int warps = 0;          // 0: the team's own
    bool streamed = false;
    bool staged = false;
    double ms = 1e300;
    bool lean = false;
};

// Tuning cache: the autotuner's choices, kept for the life of the process
// and keyed by the device, the precision, the staging setting and every
// problem's shape (frame, PSF side, stride, lattice, chains, sampler, team),
// in order.  A handle created later for the same shapes starts with the
// tuned plan instead of the automatic one.  A plan changes no chain (every
// plan gives bit-identical results), only the speed.
struct TuneEntry {
    bool one_launch = false;
    std::vector<TuneChoice> groups;
};
std::mutex g_tune_mu;
std::map<std::vector<long long>, TuneEntry> g_tune_cache;
bool g_tune_cache_on = true;

std::vector<long long> tune_key(const bdecon_handle* h)
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<long long> k = {dev, h->sms, h->precision, h->staging, h->lean};
    for (size_t q = 0; q < h->probs.size(); ++q) {
        const ProbHost& ph = h->probs[q];
        k.insert(k.end(), {ph.H, ph.W, ph.L, ph.S, ph.f, ph.p.n_chains,
                           (ph.p.flags & BDECON_FLAG_AUGMENTED) ? 1LL : 0LL, h->imgs[q].team});
    }
    return k;
}

// Apply a cached plan to a handle whose groups are formed; false if none.
bool apply_cached_plan(bdecon_handle* h)
{
    TuneEntry e;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        if (!g_tune_cache_on) return false;
        auto it = g_tune_cache.find(tune_key(h));
        if (it == g_tune_cache.end()) return false;
        e = it->second;
    }
    h->one_launch = e.one_launch;
    form_groups(h);
    if (e.groups.size() != h->groups.size()) {
        h->one_launch = false;
        form_groups(h);
        return false;
    }
    for (size_t g = 0; g < h->groups.size(); ++g) {
        h->groups[g].warps = e.groups[g].warps;
        h->groups[g].user_warps = true;
        h->groups[g].streamed = e.groups[g].streamed;
        h->groups[g].no_stage = !e.groups[g].staged;
        h->groups[g].user_stage = true;
        h->groups[g].user_lean = e.groups[g].lean ? 1 : 0;
    }
    return true;
}

bdecon_status create_impl(const bdecon_problem* ps, int n, void* stream, void* ws, size_t ws_bytes, bdecon_handle** out)
{
    if (!out) return fail(nullptr, BDECON_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!ps || n < 1) return fail(nullptr, BDECON_ERR_INVALID, "no problems");
    for (int k = 0; k < n; ++k) {
        bdecon_status s = validate(ps[k], k);
        if (s != BDECON_OK) return s;
        if (ps[k].precision != ps[0].precision)
            return fail(nullptr, BDECON_ERR_INVALID, "all problems of a batch must use the same precision");
    }
    bdecon_handle* h = new bdecon_handle();
    h->precision = ps[0].precision;
    h->st = (cudaStream_t)stream;
    h->max_sweeps = 0;
    for (int k = 0; k < n; ++k) h->max_sweeps = std::max(h->max_sweeps, ps[k].max_sweeps ? ps[k].max_sweeps : 4096);
    h->probs.resize(n);
    for (int k = 0; k < n; ++k) {
        h->probs[k].p = ps[k];
        if (h->probs[k].p.step == 0.0) h->probs[k].p.step = 0.2;
        describe(h->probs[k]);
    }
    int dev = 0;
    auto bail = [&](bdecon_status s) {
        std::string m = h->err;
        if (h->own_arena && h->arena) cudaFree(h->arena);
        delete h;
        g_err = m;
        return s;
    };
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bail(fail(h, BDECON_ERR_CUDA, "no CUDA device"));
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return bail(fail(h, BDECON_ERR_CUDA, "device does not support cooperative launches"));
    const size_t need = layout(h, h->probs, h->chh, h->precision, h->max_sweeps);
    if (ws) {
        if (ws_bytes < need) return bail(fail(h, BDECON_ERR_NOMEM, "workspace of %zu bytes, %zu needed", ws_bytes, need));
        if (((uintptr_t)ws) % 256) return bail(fail(h, BDECON_ERR_INVALID, "workspace must be 256-byte aligned"));
        h->arena = (char*)ws;
        h->own_arena = false;
    } else {
        void* p = nullptr;
        if (cudaMalloc(&p, need) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(h, BDECON_ERR_NOMEM, "cudaMalloc of %zu bytes failed", need));
        }
        h->arena = (char*)p;
        h->own_arena = true;
    }
    h->arena_bytes = need;
    if (cudaMemsetAsync(h->arena, 0, need, h->st) != cudaSuccess) return bail(fail(h, BDECON_ERR_CUDA, "memset"));
    h->d_imgs = (Image*)(h->arena + h->o_imgs);
    h->d_chains = (Chain*)(h->arena + h->o_chains);
    h->d_gchains = (Chain*)(h->arena + h->o_gchains);
    h->d_err = (int*)(h->arena + h->o_err);
    h->d_out = (double*)(h->arena + h->o_out);
    h->d_up = (double*)(h->arena + h->o_up);
    // descriptors
    h->imgs.resize(n);
    for (int k = 0; k < n; ++k) {
        ProbHost& ph = h->probs[k];
        Image& im = h->imgs[k];
        std::memset(&im, 0, sizeof im);
        im.H = ph.H; im.W = ph.W; im.L = ph.L; im.R = ph.R; im.S = ph.S; im.Ho = ph.Ho; im.Wo = ph.Wo;
        im.npi = ph.npi; im.npj = ph.npj; im.mu_pitch = ph.pitch; im.n_chains = ph.p.n_chains;
        im.seed_lo = (uint32_t)(ph.p.seed & 0xffffffffu); im.seed_hi = (uint32_t)(ph.p.seed >> 32);
        im.step = ph.p.step; im.burn_in = ph.p.burn_in; im.refresh_every = ph.p.refresh_every;
        im.n_patches = ph.n_patches; im.chain0 = ph.chain0;
        char* A = h->arena;
        im.K64 = (const double*)(A + ph.o_K64); im.K32 = (const float*)(A + ph.o_K32);
        im.f = ph.f; im.Le = ph.Le; im.Lc = ph.Lc;
        im.Ke64 = ph.f > 1 ? (const double*)(A + ph.o_Ke64) : im.K64;
        im.Ke32 = ph.f > 1 ? (const float*)(A + ph.o_Ke32) : im.K32;
        im.dat64 = (const double*)(A + ph.o_dat64); im.dat32 = (const float*)(A + ph.o_dat32);
        for (int s = 0; s < kMaxShapes; ++s) im.shape[s] = ph.shape[s];
        im.ent_kl = (const int*)(A + ph.o_ekl);
        im.ent_wa64 = (const double*)(A + ph.o_wa64); im.ent_m64 = (const double*)(A + ph.o_m64);
        im.ent_wa32 = (const float*)(A + ph.o_wa32); im.ent_m32 = (const float*)(A + ph.o_m32);
        im.tw64 = (const double*)(A + ph.o_tw64); im.tw32 = (const float*)(A + ph.o_tw32);
        im.patch_off = (const int64_t*)(A + ph.o_poff);
        im.spec_len = ph.spec_len;
        im.n_ent = (int)ph.ent_kl.size();
        im.team = problem_team(ph.Lc, ph.p.n_chains, ph.n_patches, ph.p.team_warps, h->precision == BDECON_FP32);
        ph.many = ph.p.team_warps == 0 && (long long)ph.p.n_chains * ph.n_patches >= 2048;
        im.n_tw = ph.n_tw;
        im.max_nhalf = ph.max_nhalf;
        im.sample_every = ph.p.sample_every > 0 ? ph.p.sample_every : 1;
        im.n_samples = ph.p.n_samples;
        im.adapt_fac = ph.o_adapt ? (const double*)(A + ph.o_adapt) : nullptr;
    }
    h->chains.resize(h->chh.size());
    for (int k = 0; k < n; ++k) {
        ProbHost& ph = h->probs[k];
        for (int c = 0; c < ph.p.n_chains; ++c) {
            const ChainHost& x = h->chh[ph.chain0 + c];
            Chain& ch = h->chains[ph.chain0 + c];
            std::memset(&ch, 0, sizeof ch);
            char* A = h->arena;
            const size_t nobj = (size_t)ph.Ho * ph.Wo;
            ch.img = k; ch.chain = c;
            ch.rho = A + x.o_rho; ch.mu = A + x.o_mu; ch.spec = A + x.o_spec;
            ch.cum = x.o_cum ? (float4*)(A + x.o_cum) : nullptr;
            ch.cum2 = x.o_cum2 ? (float2*)(A + x.o_cum2) : nullptr;
            ch.rho_sum = (double*)(A + ph.o_sum) + c * nobj;
            ch.rho_sq = ph.o_sq ? (double*)(A + ph.o_sq) + c * nobj : nullptr;
            ch.trace_part = (double*)(A + x.o_tpart);
            ch.acc_count = (unsigned long long*)(A + x.o_acc);
            ch.acc_log = x.o_log ? (uint8_t*)(A + x.o_log) : nullptr;
            ch.prog = (int*)(A + x.o_prog);
            ch.trace = (double*)(A + x.o_trace);
            ch.tdev = (int*)(A + x.o_tdev);
            ch.samples = ph.o_samp ? A + ph.o_samp + (h->precision == BDECON_FP32 ? 4 : 8) * nobj * ph.p.n_samples * c
                                   : nullptr;
            ch.steps = x.o_steps ? A + x.o_steps : nullptr;
            ch.phi = x.o_phi ? A + x.o_phi : nullptr;
            ch.tmap = x.o_tmap ? A + x.o_tmap : nullptr;
        }
    }
    // window-staging tensor maps (a problem without them runs unstaged plans)
    for (int k = 0; k < n; ++k) {
        ProbHost& ph = h->probs[k];
        ph.stage_ok = true;
        for (int c = 0; c < ph.p.n_chains && ph.stage_ok; ++c) {
            Chain& ch = h->chains[ph.chain0 + c];
            CUtensorMap maps[3];
            if (!ch.tmap || !encode_stage_maps(ph, ch, maps) ||
                cudaMemcpyAsync((void*)ch.tmap, maps, sizeof maps, cudaMemcpyHostToDevice, h->st) != cudaSuccess) {
                cudaGetLastError();
                ph.stage_ok = false;
            }
        }
        if (!ph.stage_ok)
            for (int c = 0; c < ph.p.n_chains; ++c) h->chains[ph.chain0 + c].tmap = nullptr;
    }
    if (cudaMemcpyAsync(h->d_imgs, h->imgs.data(), sizeof(Image) * n, cudaMemcpyHostToDevice, h->st) != cudaSuccess)
        return bail(fail(h, BDECON_ERR_CUDA, "descriptor upload"));
    // static tables (host-side index bookkeeping only)
    for (int k = 0; k < n; ++k) {
        ProbHost& ph = h->probs[k];
        if (cudaMemcpyAsync(h->arena + ph.o_ekl, ph.ent_kl.data(), 4 * ph.ent_kl.size(), cudaMemcpyHostToDevice, h->st) != cudaSuccess ||
            cudaMemcpyAsync(h->arena + ph.o_poff, ph.patch_off.data(), 8 * ph.patch_off.size(), cudaMemcpyHostToDevice, h->st) != cudaSuccess)
            return bail(fail(h, BDECON_ERR_CUDA, "table upload"));
        if (ph.o_adapt) {
            // proposal-scale factors of each burn-in sweep t: exp(g (1 - a*)) after an
            // accept, exp(-g a*) after a reject, g = 0.5 / sqrt(t)
            std::vector<double> fac(2 * (size_t)ph.p.burn_in);
            const double a = ph.p.adapt_target;
            for (int t = 1; t <= ph.p.burn_in; ++t) {
                const double g = 0.5 / std::sqrt((double)t);
                fac[2 * (t - 1)] = std::exp(g * (1.0 - a));
                fac[2 * (t - 1) + 1] = std::exp(-g * a);
            }
            if (cudaMemcpy(h->arena + ph.o_adapt, fac.data(), 8 * fac.size(), cudaMemcpyHostToDevice) != cudaSuccess)
                return bail(fail(h, BDECON_ERR_CUDA, "table upload"));
        }
        for (int c = 0; c < ph.p.n_chains; ++c) {
            const Chain& ch = h->chains[ph.chain0 + c];
            if (!ch.steps) continue;
            const int64_t nobj = (int64_t)ph.Ho * ph.Wo;
            if (h->precision == BDECON_FP32) launch_fill<float>(ch.steps, nobj, ph.p.step, h->st, &h->launches);
            else launch_fill<double>(ch.steps, nobj, ph.p.step, h->st, &h->launches);
        }
    }
    // per problem: upload inputs (host -> device), set-up kernels, initial objects, refresh
    for (int k = 0; k < n; ++k) {
        ProbHost& ph = h->probs[k];
        const bdecon_problem& p = ph.p;
        const size_t npix = (size_t)ph.H * ph.W;
        float* u_w = (float*)h->d_up;
        float* u_g = u_w + npix;
        float* u_o = u_g + npix;
        float* u_v = u_o + npix;
        double* u_psf = (double*)(u_v + npix);
        cudaError_t e = cudaMemcpyAsync(u_w, p.image, 4 * npix, cudaMemcpyHostToDevice, h->st);
        if (e == cudaSuccess && p.gain_map) e = cudaMemcpyAsync(u_g, p.gain_map, 4 * npix, cudaMemcpyHostToDevice, h->st);
        if (e == cudaSuccess && p.offset_map) e = cudaMemcpyAsync(u_o, p.offset_map, 4 * npix, cudaMemcpyHostToDevice, h->st);
        if (e == cudaSuccess && p.var_map) e = cudaMemcpyAsync(u_v, p.var_map, 4 * npix, cudaMemcpyHostToDevice, h->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(u_psf, p.psf, 8 * (size_t)ph.L * ph.L, cudaMemcpyHostToDevice, h->st);
        if (e != cudaSuccess) return bail(fail(h, BDECON_ERR_CUDA, "input upload: %s", cudaGetErrorString(e)));
        double* scr = (double*)(h->arena + ph.o_scr);
        double* b0 = h->d_out;
        launch_setup(h->imgs[k], h->d_imgs + k, u_w, p.gain_map ? u_g : nullptr, p.offset_map ? u_o : nullptr,
                     p.var_map ? u_v : nullptr, p.gain, p.offset, p.read_var, u_psf, b0, scr, h->st, &h->launches);
        for (int c = 0; c < p.n_chains; ++c) {
            const Chain& ch = h->chains[ph.chain0 + c];
            if (h->precision == BDECON_FP32) launch_init_rho<float>(h->imgs[k], ch, b0, h->st, &h->launches);
            else launch_init_rho<double>(h->imgs[k], ch, b0, h->st, &h->launches);
        }
        // the staging buffer is reused by the next problem: finish this one first
        if (cudaStreamSynchronize(h->st) != cudaSuccess) return bail(fail(h, BDECON_ERR_CUDA, "set-up: %s", cudaGetErrorString(cudaGetLastError())));
        for (int c = 0; c < p.n_chains; ++c) {
            const Chain& ch = h->chains[ph.chain0 + c];
            if (refresh(h, ph.chain0 + c, 1, ch.trace) != BDECON_OK) return bail(BDECON_ERR_CUDA);
            if (ch.phi) {
                // augmented sampler: photon counts drawn at the initial mu (uniforms
                // of sweep 0), then the trace starts at the joint density
                if (h->precision == BDECON_FP32) launch_sample_phi<float>(h->imgs[k], ch, 0, h->d_err, h->st, &h->launches);
                else launch_sample_phi<double>(h->imgs[k], ch, 0, h->d_err, h->st, &h->launches);
                if (refresh(h, ph.chain0 + c, 1, ch.trace) != BDECON_OK) return bail(BDECON_ERR_CUDA);
            }
        }
    }
    form_groups(h);
    // the autotuner's plan for these shapes, if one was tuned in this process
    const bool cached = apply_cached_plan(h);
    bdecon_status s = make_plan(h);
    if (s != BDECON_OK && cached) {
        h->one_launch = false;
        form_groups(h);
        s = make_plan(h);
    }
    if (s != BDECON_OK) return bail(s);
    s = check_device(h);
    if (s != BDECON_OK) return bail(s);
    *out = h;
    return BDECON_OK;
}


// A launch over one or more handles (all of one precision on one device):
// the groups, the host copy of the launch's chain table (group order), the
// owning handle of each chain, and the device tables the kernel reads.
struct LaunchSet {
    std::vector<bdecon_handle*> hs;
    std::vector<Group> groups;
    std::vector<Chain> gch;
    std::vector<int> owner;
    const Image* d_imgs = nullptr;
    Chain* d_gch = nullptr;
};

void own_launch_set(bdecon_handle* h, LaunchSet& ls)
{
    ls.hs.assign(1, h);
    ls.groups = h->groups;
    ls.gch = h->gch;
    ls.owner.assign(h->gch.size(), 0);
    ls.d_imgs = h->d_imgs;
    ls.d_gch = h->d_gchains;
}

// Longest segment <= want, starting after sweep t0, that crosses no
// problem's refresh boundary.
int segment_len_at(const bdecon_handle* h, int64_t t0, int want)
{
    int len = std::min(want, kMaxSlots);
    for (const auto& ph : h->probs)
        if (ph.p.refresh_every > 0)
            len = (int)std::min<int64_t>(len, (t0 / ph.p.refresh_every + 1) * ph.p.refresh_every - t0);
    return len;
}

int segment_len(const bdecon_handle* h, int want)
{
    return segment_len_at(h, h->sweeps, want);
}

// Host bookkeeping of a finished segment: sweep counter and running-mean count.
void advance_host(bdecon_handle* h, int len)
{
    const int64_t t0 = h->sweeps;
    h->sweeps += len;
    for (auto& ph : h->probs)
        for (int64_t t = t0 + 1; t <= t0 + len; ++t)
            if (t > ph.p.burn_in) ++ph.n_sum;
}

// After a segment: trace, counters, running-sum bookkeeping, refreshes.
bdecon_status finish_segment(bdecon_handle* h, int len)
{
    launch_trace(h->d_imgs, h->d_chains, (int)h->chains.size(), len, h->st, &h->launches);
    CK(h, cudaGetLastError());
    advance_host(h, len);
    for (auto& ph : h->probs) {
        if (ph.p.refresh_every > 0 && h->sweeps % ph.p.refresh_every == 0)
            for (int c = 0; c < ph.p.n_chains; ++c) {
                const int ci = ph.chain0 + c;
                bdecon_status s = refresh(h, ci, 1, h->chains[ci].trace, h->chains[ci].tdev);
                if (s != BDECON_OK) return s;
            }
    }
    return BDECON_OK;
}

// One segment of len sweeps over every handle of the launch set, on stream st
// (kernel launches only: each chain starts from its own device sweep
// counter, so the segment can be captured in a CUDA graph); eh receives
// errors; gev (optional) gets an event before each group's launch and after
// the last.  lens (optional): sweeps of each handle's chains, at most len;
// the chain table must then carry them (Chain::n_sweeps).
bdecon_status run_segment(LaunchSet& ls, int len, cudaStream_t st, bdecon_handle* eh, cudaEvent_t* gev = nullptr,
                          const int* lens = nullptr)
{
    for (size_t hi = 0; hi < ls.hs.size(); ++hi) {
        bdecon_handle* h = ls.hs[hi];
        launch_reset(h->d_imgs, h->d_chains, (int)h->chains.size(), lens ? lens[hi] : len, st, &h->launches);
    }
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (eh->timing) {
        if (eh->ev_used + 2 > eh->ev_pool.size()) {
            for (int k = 0; k < 2; ++k) {
                cudaEvent_t ev;
                CK(eh, cudaEventCreate(&ev));
                eh->ev_pool.push_back(ev);
            }
        }
        ev0 = eh->ev_pool[eh->ev_used];
        ev1 = eh->ev_pool[eh->ev_used + 1];
        eh->ev_used += 2;
        CK(eh, cudaEventRecord(ev0, st));
    }
    for (size_t gi = 0; gi < ls.groups.size(); ++gi) {
        const Group& g = ls.groups[gi];
        if (gev) CK(eh, cudaEventRecord(gev[gi], st));
        SweepArgs a;
        a.imgs = ls.d_imgs; a.chains = ls.d_gch + g.chain_off; a.n_chains = g.n_chains;
        a.n_sweeps = len; a.err = eh->d_err; a.resident = g.resident;
        a.wait_ns = eh->wait_ns; a.silent_block = gi == 0 ? eh->silent_block : -1;
        a.aug = g.aug ? 1 : 0;
        a.fine = g.fine ? 1 : 0;
        a.solo = g.solo ? 1 : 0;
        a.stage = g.stage;
        a.lean = g.lean ? 1 : 0;
        cudaError_t e = eh->precision == BDECON_FP32 ? launch_sweep<float>(a, g.grid, g.threads, g.smem, st)
                                                     : launch_sweep<double>(a, g.grid, g.threads, g.smem, st);
        if (e != cudaSuccess)
            return fail(eh, BDECON_ERR_CUDA, "sweep launch (%d blocks x %d threads, %zu B shared): %s", g.grid,
                        g.threads, g.smem, cudaGetErrorString(e));
        ++eh->launches;
    }
    if (gev) CK(eh, cudaEventRecord(gev[ls.groups.size()], st));
    if (eh->timing) CK(eh, cudaEventRecord(ev1, st));
    for (size_t hi = 0; hi < ls.hs.size(); ++hi) {
        bdecon_status s = finish_segment(ls.hs[hi], lens ? lens[hi] : len);
        if (s != BDECON_OK) return s;
    }
    return BDECON_OK;
}

// The segment sequence of n sweeps from the current counter: each segment's
// length, followed by -1-k for each problem k refreshed after it.
std::vector<int> sweep_signature(const bdecon_handle* h, int n)
{
    std::vector<int> sig;
    int64_t sw = h->sweeps;
    while (n > 0) {
        const int len = segment_len_at(h, sw, n);
        sig.push_back(len);
        sw += len;
        for (size_t k = 0; k < h->probs.size(); ++k) {
            const int re = h->probs[k].p.refresh_every;
            if (re > 0 && sw % re == 0) sig.push_back(-1 - (int)k);
        }
        n -= len;
    }
    return sig;
}

// n sweeps as one CUDA-graph launch: the kernels of every segment (reset,
// sweep launches, trace, refreshes) are captured once per segment sequence
// and replayed; the host only advances its counters.
bdecon_status graph_sweep(bdecon_handle* h, int n)
{
    const std::vector<int> sig = sweep_signature(h, n);
    bdecon_handle::GraphEntry* ge = nullptr;
    for (auto& g : h->graphs)
        if (g.sig == sig) ge = &g;
    if (!ge) {
        if (!h->cap_st) CK(h, cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking));
        const int64_t sw0 = h->sweeps, l0 = h->launches;
        std::vector<int64_t> nsum0;
        for (const auto& ph : h->probs) nsum0.push_back(ph.n_sum);
        const cudaStream_t user_st = h->st;
        const bool timing = h->timing;
        h->st = h->cap_st;
        h->timing = false;
        bdecon_status s = BDECON_OK;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            LaunchSet ls;
            own_launch_set(h, ls);
            for (int left = n; left > 0 && s == BDECON_OK;) {
                const int len = segment_len(h, left);
                s = run_segment(ls, len, h->cap_st, h);
                left -= len;
            }
            e = cudaStreamEndCapture(h->cap_st, &graph);
        }
        h->st = user_st;
        h->timing = timing;
        h->sweeps = sw0;
        for (size_t k = 0; k < h->probs.size(); ++k) h->probs[k].n_sum = nsum0[k];
        const int64_t nl = h->launches - l0;
        h->launches = l0;
        if (s != BDECON_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (e != cudaSuccess) return fail(h, BDECON_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(h, BDECON_ERR_CUDA, "graph instantiation: %s", cudaGetErrorString(e));
        if (h->graphs.size() >= 8) {
            cudaGraphExecDestroy(h->graphs.front().exec);
            h->graphs.erase(h->graphs.begin());
        }
        h->graphs.push_back({sig, exec, nl});
        ge = &h->graphs.back();
    }
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (h->timing) {
        if (h->ev_used + 2 > h->ev_pool.size())
            for (int k = 0; k < 2; ++k) {
                cudaEvent_t ev;
                CK(h, cudaEventCreate(&ev));
                h->ev_pool.push_back(ev);
            }
        ev0 = h->ev_pool[h->ev_used];
        ev1 = h->ev_pool[h->ev_used + 1];
        h->ev_used += 2;
        CK(h, cudaEventRecord(ev0, h->st));
    }
    CK(h, cudaGraphLaunch(ge->exec, h->st));
    if (h->timing) CK(h, cudaEventRecord(ev1, h->st));
    h->launches += ge->launches;
    for (int x : sig)
        if (x > 0) advance_host(h, x);
    return BDECON_OK;
}

bdecon_status chain_index(bdecon_handle* h, int p, int c, int* ci)
{
    if (p < 0 || p >= (int)h->probs.size()) return fail(h, BDECON_ERR_INVALID, "problem index %d", p);
    if (c < 0 || c >= h->probs[p].p.n_chains) return fail(h, BDECON_ERR_INVALID, "chain index %d", c);
    *ci = h->probs[p].chain0 + c;
    return BDECON_OK;
}

}  // namespace

// =================================================================== C ABI

extern "C" {

bdecon_status bdecon_workspace_size(const bdecon_problem* ps, int32_t n, size_t* bytes)
{
    if (!ps || n < 1 || !bytes) return fail(nullptr, BDECON_ERR_INVALID, "bad arguments");
    for (int k = 0; k < n; ++k) {
        bdecon_status s = validate(ps[k], k);
        if (s != BDECON_OK) return s;
    }
    bdecon_handle tmp;
    std::vector<ProbHost> probs(n);
    int ms = 0;
    for (int k = 0; k < n; ++k) {
        probs[k].p = ps[k];
        describe(probs[k]);
        ms = std::max(ms, ps[k].max_sweeps ? ps[k].max_sweeps : 4096);
    }
    std::vector<ChainHost> chh;
    *bytes = layout(&tmp, probs, chh, ps[0].precision, ms);
    return BDECON_OK;
}

bdecon_status bdecon_create(const bdecon_problem* p, void* stream, bdecon_handle** out)
{
    return create_impl(p, 1, stream, nullptr, 0, out);
}

bdecon_status bdecon_batch_create(const bdecon_problem* ps, int32_t n, void* stream, bdecon_handle** out)
{
    return create_impl(ps, n, stream, nullptr, 0, out);
}

bdecon_status bdecon_create_in(const bdecon_problem* ps, int32_t n, void* stream, void* ws, size_t bytes,
                               bdecon_handle** out)
{
    if (!ws) return fail(nullptr, BDECON_ERR_INVALID, "workspace is NULL");
    return create_impl(ps, n, stream, ws, bytes, out);
}

void bdecon_destroy(bdecon_handle* h)
{
    if (!h) return;
    if (h->st) cudaStreamSynchronize(h->st); else cudaDeviceSynchronize();
    drop_graphs(h);
    if (h->cap_st) cudaStreamDestroy(h->cap_st);
    for (cudaEvent_t ev : h->ev_pool) cudaEventDestroy(ev);
    if (h->own_arena && h->arena) cudaFree(h->arena);
    delete h;
}

const char* bdecon_last_error(const bdecon_handle* h)
{
    return h ? h->err.c_str() : g_err.c_str();
}

bdecon_status bdecon_sweep(bdecon_handle* h, int32_t n)
{
    if (!h) return fail(nullptr, BDECON_ERR_INVALID, "handle is NULL");
    if (h->failed) return fail(h, BDECON_ERR_STATE, "handle failed earlier: %s", h->err.c_str());
    if (n < 0) return fail(h, BDECON_ERR_INVALID, "negative sweep count");
    if (h->sweeps + n > h->max_sweeps)
        return fail(h, BDECON_ERR_INVALID, "trace capacity %d exceeded (%lld + %d sweeps)", h->max_sweeps,
                    (long long)h->sweeps, n);
    if (h->use_graph && n > 0) return graph_sweep(h, n);
    LaunchSet ls;
    own_launch_set(h, ls);
    while (n > 0) {
        const int len = segment_len(h, n);
        bdecon_status s = run_segment(ls, len, h->st, h);
        if (s != BDECON_OK) return s;
        n -= len;
    }
    return BDECON_OK;
}

bdecon_status bdecon_set_graph(bdecon_handle* h, int32_t enable)
{
    if (!h) return fail(nullptr, BDECON_ERR_INVALID, "handle is NULL");
    bdecon_status s = check_device(h);
    if (s != BDECON_OK) return s;
    h->use_graph = enable != 0;
    if (!h->use_graph) drop_graphs(h);
    return BDECON_OK;
}

bdecon_status bdecon_sync(bdecon_handle* h)
{
    if (!h) return fail(nullptr, BDECON_ERR_INVALID, "handle is NULL");
    return check_device(h);
}

bdecon_status bdecon_posterior_mean(bdecon_handle* h, int32_t p, double* out, int32_t crop)
{
    if (!h || !out) return fail(h, BDECON_ERR_INVALID, "bad arguments");
    int ci;
    bdecon_status s = chain_index(h, p, 0, &ci);
    if (s != BDECON_OK) return s;
    ProbHost& ph = h->probs[p];
    if (ph.n_sum == 0) return fail(h, BDECON_ERR_STATE, "no sweep after burn-in yet");
    const int oh = crop ? ph.f * ph.H : ph.Ho, ow = crop ? ph.f * ph.W : ph.Wo;
    launch_mean(h->chains[ci].rho_sum, ph.p.n_chains, (int64_t)ph.Ho * ph.Wo, ph.Ho, ph.Wo, crop ? ph.R : 0, oh, ow,
                1.0 / ((double)ph.n_sum * ph.p.n_chains), h->d_up, nullptr, 0, h->st, &h->launches);
    CK(h, cudaMemcpyAsync(out, h->d_up, 8 * (size_t)oh * ow, cudaMemcpyDeviceToHost, h->st));
    return check_device(h);
}

namespace {

// Pooled map of kind 0..3 (mean, variance, std, cv) into host out.
bdecon_status pooled_map(bdecon_handle* h, int32_t p, double* out, int32_t crop, int kind)
{
    if (!h || !out) return fail(h, BDECON_ERR_INVALID, "bad arguments");
    int ci;
    bdecon_status s = chain_index(h, p, 0, &ci);
    if (s != BDECON_OK) return s;
    ProbHost& ph = h->probs[p];
    if (kind > 0 && !ph.o_sq) return fail(h, BDECON_ERR_STATE, "created without BDECON_FLAG_SECOND_MOMENT");
    if (ph.n_sum == 0) return fail(h, BDECON_ERR_STATE, "no sweep after burn-in yet");
    const int oh = crop ? ph.f * ph.H : ph.Ho, ow = crop ? ph.f * ph.W : ph.Wo;
    launch_mean(h->chains[ci].rho_sum, ph.p.n_chains, (int64_t)ph.Ho * ph.Wo, ph.Ho, ph.Wo, crop ? ph.R : 0, oh, ow,
                1.0 / ((double)ph.n_sum * ph.p.n_chains), h->d_up, h->chains[ci].rho_sq, kind, h->st, &h->launches);
    CK(h, cudaMemcpyAsync(out, h->d_up, 8 * (size_t)oh * ow, cudaMemcpyDeviceToHost, h->st));
    return check_device(h);
}

// Kept-object slots of problem p filled so far: [first, first + count).
void kept_range(const bdecon_handle* h, const ProbHost& ph, int& first, int& count)
{
    const int every = ph.p.sample_every > 0 ? ph.p.sample_every : 1;
    const int64_t past = h->sweeps - ph.p.burn_in;
    const int64_t filled = past > 0 ? std::min<int64_t>(past / every, ph.p.n_samples) : 0;
    first = (int)std::min<int64_t>(ph.samp_first, filled);
    count = (int)filled - first;
}

}  // namespace

bdecon_status bdecon_posterior_var(bdecon_handle* h, int32_t p, double* out, int32_t crop)
{
    return pooled_map(h, p, out, crop, 1);
}

bdecon_status bdecon_posterior_std(bdecon_handle* h, int32_t p, double* out, int32_t crop)
{
    return pooled_map(h, p, out, crop, 2);
}

bdecon_status bdecon_posterior_cv(bdecon_handle* h, int32_t p, double* out, int32_t crop)
{
    return pooled_map(h, p, out, crop, 3);
}

bdecon_status bdecon_get_samples(bdecon_handle* h, int32_t p, int32_t c, double* out, size_t cap, size_t* n)
{
    if (!h || !n) return fail(h, BDECON_ERR_INVALID, "bad arguments");
    int ci;
    bdecon_status s = chain_index(h, p, c, &ci);
    if (s != BDECON_OK) return s;
    const ProbHost& ph = h->probs[p];
    int first, count;
    kept_range(h, ph, first, count);
    const size_t nobj = (size_t)ph.Ho * ph.Wo;
    *n = (size_t)count * nobj;
    if (out && cap) {
        const size_t ts = h->precision == BDECON_FP32 ? 4 : 8;
        for (int k = 0; k < count && (size_t)(k + 1) * nobj <= cap; ++k) {
            const char* src = (const char*)h->chains[ci].samples + ts * nobj * (size_t)(first + k);
            if (h->precision == BDECON_FP32) launch_convert<float>(src, h->d_up, (int64_t)nobj, ph.Ho, ph.Wo, ph.Wo, h->st, &h->launches);
            else launch_convert<double>(src, h->d_up, (int64_t)nobj, ph.Ho, ph.Wo, ph.Wo, h->st, &h->launches);
            CK(h, cudaMemcpyAsync(out + (size_t)k * nobj, h->d_up, 8 * nobj, cudaMemcpyDeviceToHost, h->st));
        }
    }
    return check_device(h);
}

bdecon_status bdecon_posterior_quantiles(bdecon_handle* h, int32_t p, const double* q, int32_t nq, double* out,
                                         int32_t crop)
{
    if (!h || !q || !out) return fail(h, BDECON_ERR_INVALID, "bad arguments");
    if (nq < 1 || nq > kMaxQuantiles) return fail(h, BDECON_ERR_INVALID, "nq must be 1..%d", kMaxQuantiles);
    for (int k = 0; k < nq; ++k)
        if (!(q[k] >= 0.0 && q[k] <= 1.0)) return fail(h, BDECON_ERR_INVALID, "q[%d] must be in [0, 1]", k);
    int ci;
    bdecon_status s = chain_index(h, p, 0, &ci);
    if (s != BDECON_OK) return s;
    const ProbHost& ph = h->probs[p];
    if (!ph.o_samp) return fail(h, BDECON_ERR_STATE, "created with n_samples = 0");
    int first, count;
    kept_range(h, ph, first, count);
    if (count < 1) return fail(h, BDECON_ERR_STATE, "no object kept yet");
    if ((int64_t)count * ph.p.n_chains > kMaxQuantileValues)
        return fail(h, BDECON_ERR_INVALID, "%d kept values per pixel, at most %d", count * ph.p.n_chains, kMaxQuantileValues);
    s = check_device(h);
    if (s != BDECON_OK) return s;
    const int oh = crop ? ph.f * ph.H : ph.Ho, ow = crop ? ph.f * ph.W : ph.Wo;
    const int64_t npix = (int64_t)oh * ow, nobj = (int64_t)ph.Ho * ph.Wo;
    // staging in d_up: the probabilities, then nq values per pixel of a chunk
    double* dq = h->d_up;
    double* dout = h->d_up + kMaxQuantiles;
    const int64_t chunk = ((int64_t)(h->up_bytes / 8) - kMaxQuantiles) / nq;
    if (chunk < 1) return fail(h, BDECON_ERR_NOMEM, "staging buffer too small");
    CK(h, cudaMemcpyAsync(dq, q, 8 * (size_t)nq, cudaMemcpyHostToDevice, h->st));
    const int64_t cstride = nobj * ph.p.n_samples;
    for (int64_t p0 = 0; p0 < npix; p0 += chunk) {
        const int64_t np = std::min(chunk, npix - p0);
        cudaError_t e = h->precision == BDECON_FP32
                            ? launch_quantiles<float>(h->chains[ci].samples, cstride, ph.p.n_chains, first, count, nobj,
                                                      ph.Wo, crop ? ph.R : 0, ow, p0, np, dq, nq, dout, h->st, &h->launches)
                            : launch_quantiles<double>(h->chains[ci].samples, cstride, ph.p.n_chains, first, count, nobj,
                                                       ph.Wo, crop ? ph.R : 0, ow, p0, np, dq, nq, dout, h->st, &h->launches);
        if (e != cudaSuccess) return fail(h, BDECON_ERR_CUDA, "quantile kernel: %s", cudaGetErrorString(e));
        for (int k = 0; k < nq; ++k)
            CK(h, cudaMemcpyAsync(out + (size_t)k * npix + p0, dout + (size_t)k * np, 8 * (size_t)np,
                                  cudaMemcpyDeviceToHost, h->st));
        CK(h, cudaStreamSynchronize(h->st));   // the staging buffer is reused by the next chunk
    }
    return check_device(h);
}

bdecon_status bdecon_log_posterior_trace(bdecon_handle* h, int32_t p, int32_t c, double* out, size_t cap, size_t* n)
{
    if (!h || !n) return fail(h, BDECON_ERR_INVALID, "bad arguments");
    int ci;
    bdecon_status s = chain_index(h, p, c, &ci);
    if (s != BDECON_OK) return s;
    *n = (size_t)h->sweeps;
    if (out && cap) {
        const size_t k = std::min(cap, (size_t)h->sweeps);
        CK(h, cudaMemcpyAsync(out, h->chains[ci].trace + 1, 8 * k, cudaMemcpyDeviceToHost, h->st));
    }
    return check_device(h);
}

bdecon_status bdecon_accept_counts(bdecon_handle* h, int32_t p, int32_t c, int64_t* out, size_t cap, size_t* n)
{
    if (!h || !n) return fail(h, BDECON_ERR_INVALID, "bad arguments");
    int ci;
    bdecon_status s = chain_index(h, p, c, &ci);
    if (s != BDECON_OK) return s;
    *n = (size_t)h->sweeps;
    if (out && cap) {
        const size_t k = std::min(cap, (size_t)h->sweeps);
        CK(h, cudaMemcpyAsync(out, h->chains[ci].acc_count, 8 * k, cudaMemcpyDeviceToHost, h->st));
    }
    return check_device(h);
}

bdecon_status bdecon_accept_log(bdecon_handle* h, int32_t p, int32_t c, uint8_t* out, size_t cap, size_t* n)
{
    if (!h || !n) return fail(h, BDECON_ERR_INVALID, "bad arguments");
    int ci;
    bdecon_status s = chain_index(h, p, c, &ci);
    if (s != BDECON_OK) return s;
    if (!h->chains[ci].acc_log) return fail(h, BDECON_ERR_STATE, "created without BDECON_FLAG_ACCEPT_LOG");
    const ProbHost& ph = h->probs[p];
    *n = (size_t)h->sweeps * ph.Ho * ph.Wo;
    if (out && cap) CK(h, cudaMemcpyAsync(out, h->chains[ci].acc_log, std::min(cap, *n), cudaMemcpyDeviceToHost, h->st));
    return check_device(h);
}

bdecon_status bdecon_get_state(bdecon_handle* h, int32_t p, int32_t c, double* rho, int64_t* sweeps)
{
    if (!h) return fail(nullptr, BDECON_ERR_INVALID, "handle is NULL");
    int ci;
    bdecon_status s = chain_index(h, p, c, &ci);
    if (s != BDECON_OK) return s;
    const ProbHost& ph = h->probs[p];
    if (sweeps) *sweeps = h->sweeps;
    if (rho) {
        const int64_t n = (int64_t)ph.Ho * ph.Wo;
        if (h->precision == BDECON_FP32) launch_convert<float>(h->chains[ci].rho, h->d_up, n, ph.Ho, ph.Wo, ph.Wo, h->st, &h->launches);
        else launch_convert<double>(h->chains[ci].rho, h->d_up, n, ph.Ho, ph.Wo, ph.Wo, h->st, &h->launches);
        CK(h, cudaMemcpyAsync(rho, h->d_up, 8 * (size_t)n, cudaMemcpyDeviceToHost, h->st));
    }
    return check_device(h);
}

bdecon_status bdecon_get_steps(bdecon_handle* h, int32_t p, int32_t c, double* out)
{
    if (!h || !out) return fail(h, BDECON_ERR_INVALID, "bad arguments");
    int ci;
    bdecon_status s = chain_index(h, p, c, &ci);
    if (s != BDECON_OK) return s;
    const ProbHost& ph = h->probs[p];
    const int64_t n = (int64_t)ph.Ho * ph.Wo;
    const Chain& ch = h->chains[ci];
    if (ch.steps) {
        if (h->precision == BDECON_FP32) launch_convert<float>(ch.steps, h->d_up, n, ph.Ho, ph.Wo, ph.Wo, h->st, &h->launches);
        else launch_convert<double>(ch.steps, h->d_up, n, ph.Ho, ph.Wo, ph.Wo, h->st, &h->launches);
        CK(h, cudaMemcpyAsync(out, h->d_up, 8 * (size_t)n, cudaMemcpyDeviceToHost, h->st));
    } else {
        for (int64_t k = 0; k < n; ++k) out[k] = ph.p.step;
    }
    return check_device(h);
}

bdecon_status bdecon_get_phi(bdecon_handle* h, int32_t p, int32_t c, double* out)
{
    if (!h || !out) return fail(h, BDECON_ERR_INVALID, "bad arguments");
    int ci;
    bdecon_status s = chain_index(h, p, c, &ci);
    if (s != BDECON_OK) return s;
    const ProbHost& ph = h->probs[p];
    const Chain& ch = h->chains[ci];
    if (!ch.phi) return fail(h, BDECON_ERR_STATE, "not an augmented problem (BDECON_FLAG_AUGMENTED)");
    const int64_t n = (int64_t)ph.H * ph.W;
    if (h->precision == BDECON_FP32) launch_convert<float>(ch.phi, h->d_up, n, ph.H, ph.W, ph.pitch, h->st, &h->launches);
    else launch_convert<double>(ch.phi, h->d_up, n, ph.H, ph.W, ph.pitch, h->st, &h->launches);
    CK(h, cudaMemcpyAsync(out, h->d_up, 8 * (size_t)n, cudaMemcpyDeviceToHost, h->st));
    return check_device(h);
}

bdecon_status bdecon_get_mu(bdecon_handle* h, int32_t p, int32_t c, double* mu)
{
    if (!h || !mu) return fail(h, BDECON_ERR_INVALID, "bad arguments");
    int ci;
    bdecon_status s = chain_index(h, p, c, &ci);
    if (s != BDECON_OK) return s;
    const ProbHost& ph = h->probs[p];
    const int64_t n = (int64_t)ph.H * ph.W;
    if (h->precision == BDECON_FP32) launch_convert<float>(h->chains[ci].mu, h->d_up, n, ph.H, ph.W, ph.pitch, h->st, &h->launches);
    else launch_convert<double>(h->chains[ci].mu, h->d_up, n, ph.H, ph.W, ph.pitch, h->st, &h->launches);
    CK(h, cudaMemcpyAsync(mu, h->d_up, 8 * (size_t)n, cudaMemcpyDeviceToHost, h->st));
    return check_device(h);
}

bdecon_status bdecon_set_state(bdecon_handle* h, int32_t p, int32_t c, const double* rho, int64_t sweeps)
{
    if (!h || !rho) return fail(h, BDECON_ERR_INVALID, "bad arguments");
    int ci;
    bdecon_status s = chain_index(h, p, c, &ci);
    if (s != BDECON_OK) return s;
    if (sweeps < 0 || sweeps > h->max_sweeps) return fail(h, BDECON_ERR_INVALID, "sweep counter %lld out of range", (long long)sweeps);
    const ProbHost& ph0 = h->probs[p];
    const int64_t n = (int64_t)ph0.Ho * ph0.Wo;
    for (int64_t k = 0; k < n; ++k)
        if (!(std::isfinite(rho[k]) && rho[k] > 0.0)) return fail(h, BDECON_ERR_INVALID, "rho[%lld] must be finite and > 0", (long long)k);
    s = check_device(h);
    if (s != BDECON_OK) return s;
    CK(h, cudaMemcpyAsync(h->d_up, rho, 8 * (size_t)n, cudaMemcpyHostToDevice, h->st));
    if (h->precision == BDECON_FP32) launch_set_rho<float>(h->d_up, h->chains[ci].rho, n, h->st, &h->launches);
    else launch_set_rho<double>(h->d_up, h->chains[ci].rho, n, h->st, &h->launches);
    h->sweeps = sweeps;
    // the sweep counter is shared by every chain of the handle: rebase all traces
    launch_set_counters(h->d_chains, (int)h->chains.size(), (int)sweeps, h->st, &h->launches);
    for (size_t k = 0; k < h->chains.size(); ++k) {
        s = refresh(h, (int)k, 1, h->chains[k].trace + sweeps);
        if (s != BDECON_OK) return s;
    }
    for (auto& ph : h->probs) {
        ph.n_sum = 0;
        {   // objects kept before the resume point are not this run's
            const int every = ph.p.sample_every > 0 ? ph.p.sample_every : 1;
            const int64_t past = sweeps - ph.p.burn_in;
            ph.samp_first = past > 0 ? (int)std::min<int64_t>(past / every, ph.p.n_samples) : 0;
        }
        for (int k = 0; k < ph.p.n_chains; ++k) {
            const Chain& ch = h->chains[ph.chain0 + k];
            CK(h, cudaMemsetAsync(ch.rho_sum, 0, 8 * (size_t)ph.Ho * ph.Wo, h->st));
            if (ch.rho_sq) CK(h, cudaMemsetAsync(ch.rho_sq, 0, 8 * (size_t)ph.Ho * ph.Wo, h->st));
        }
    }
    return check_device(h);
}

bdecon_status bdecon_log_posterior(bdecon_handle* h, int32_t p, int32_t c, double* out)
{
    if (!h || !out) return fail(h, BDECON_ERR_INVALID, "bad arguments");
    int ci;
    bdecon_status s = chain_index(h, p, c, &ci);
    if (s != BDECON_OK) return s;
    s = refresh(h, ci, 0, h->d_out);
    if (s != BDECON_OK) return s;
    CK(h, cudaMemcpyAsync(out, h->d_out, 8, cudaMemcpyDeviceToHost, h->st));
    return check_device(h);
}

bdecon_status bdecon_delta(bdecon_handle* h, int32_t p, int32_t c, int64_t m, double rho_new, double* dL, double* dP,
                           int32_t* ok)
{
    if (!h || !dL || !dP || !ok) return fail(h, BDECON_ERR_INVALID, "bad arguments");
    int ci;
    bdecon_status s = chain_index(h, p, c, &ci);
    if (s != BDECON_OK) return s;
    const ProbHost& ph = h->probs[p];
    if (m < 0 || m >= (int64_t)ph.Ho * ph.Wo) return fail(h, BDECON_ERR_INVALID, "pixel %lld out of range", (long long)m);
    if (!(std::isfinite(rho_new) && rho_new > 0.0)) return fail(h, BDECON_ERR_INVALID, "rho_new must be finite and > 0");
    if (ph.p.flags & BDECON_FLAG_AUGMENTED)
        return fail(h, BDECON_ERR_STATE, "bdecon_delta evaluates Eq. 6; not available for augmented problems");
    if (h->precision == BDECON_FP32) launch_delta<float>(h->d_imgs + p, h->d_chains + ci, m, rho_new, h->d_out, h->imgs[p].team, h->st, &h->launches);
    else launch_delta<double>(h->d_imgs + p, h->d_chains + ci, m, rho_new, h->d_out, h->imgs[p].team, h->st, &h->launches);
    CK(h, cudaGetLastError());
    double r[3];
    CK(h, cudaMemcpyAsync(r, h->d_out, sizeof r, cudaMemcpyDeviceToHost, h->st));
    s = check_device(h);
    if (s != BDECON_OK) return s;
    *dL = r[0]; *dP = r[1]; *ok = r[2] != 0.0;
    return BDECON_OK;
}

bdecon_status bdecon_set_plan(bdecon_handle* h, int32_t p, int32_t tile_i, int32_t tile_j, int32_t warps)
{
    if (!h) return fail(nullptr, BDECON_ERR_INVALID, "handle is NULL");
    if (p < 0 || p >= (int)h->probs.size()) return fail(h, BDECON_ERR_INVALID, "problem index %d", p);
    ProbHost& ph = h->probs[p];
    Group& g = h->groups[h->prob_group[p]];
    const int old_i = ph.tpi, old_j = ph.tpj, old_w = g.warps;
    const bool old_u = ph.user_plan, old_uw = g.user_warps;
    if (tile_i < 0 || tile_j < 0 || warps < 0 || warps > 8) return fail(h, BDECON_ERR_INVALID, "bad plan");
    if (tile_i == 0 || tile_j == 0) {
        ph.user_plan = false;
    } else {
        ph.user_plan = true;
        ph.tpi = std::min(tile_i, ph.npi);
        ph.tpj = std::min(tile_j, ph.npj);
    }
    if (warps == 0) {
        g.user_warps = false;
    } else {
        g.warps = warps;
        g.user_warps = true;
    }
    bdecon_status s = check_device(h);
    if (s == BDECON_OK) s = make_plan(h);
    if (s != BDECON_OK) {
        ph.tpi = old_i; ph.tpj = old_j; g.warps = old_w; ph.user_plan = old_u; g.user_warps = old_uw;
        std::string m = h->err;
        make_plan(h);
        h->err = m;
    }
    return s;
}

bdecon_status bdecon_set_grouping(bdecon_handle* h, int32_t one_launch)
{
    if (!h) return fail(nullptr, BDECON_ERR_INVALID, "handle is NULL");
    bdecon_status s = check_device(h);
    if (s != BDECON_OK) return s;
    const bool old = h->one_launch;
    const std::vector<Group> old_groups = h->groups;
    const std::vector<int> old_pg = h->prob_group;
    h->one_launch = one_launch != 0;
    form_groups(h);
    s = make_plan(h);
    if (s != BDECON_OK) {
        const std::string m = h->err;
        h->one_launch = old;
        h->groups = old_groups;
        h->prob_group = old_pg;
        make_plan(h);
        h->err = m;
    }
    return s;
}

bdecon_status bdecon_set_staging(bdecon_handle* h, int32_t enable)
{
    if (!h) return fail(nullptr, BDECON_ERR_INVALID, "handle is NULL");
    bdecon_status s = check_device(h);
    if (s != BDECON_OK) return s;
    const int old = h->staging;
    const std::vector<Group> old_groups = h->groups;
    h->staging = enable != 0 ? 1 : 0;
    for (auto& g : h->groups) g.user_stage = false;
    s = make_plan(h);
    if (s != BDECON_OK) {
        const std::string m = h->err;
        h->staging = old;
        h->groups = old_groups;
        make_plan(h);
        h->err = m;
    }
    return s;
}

bdecon_status bdecon_get_staging(bdecon_handle* h, int32_t p, int32_t* staged)
{
    if (!h || !staged) return fail(h, BDECON_ERR_INVALID, "bad arguments");
    if (p < 0 || p >= (int)h->probs.size()) return fail(h, BDECON_ERR_INVALID, "problem index %d", p);
    *staged = h->groups[h->prob_group[p]].stage;
    return BDECON_OK;
}

bdecon_status bdecon_set_lean(bdecon_handle* h, int32_t mode)
{
    if (!h) return fail(nullptr, BDECON_ERR_INVALID, "handle is NULL");
    if (mode < -1 || mode > 1) return fail(h, BDECON_ERR_INVALID, "lean mode %d (-1, 0 or 1)", mode);
    bdecon_status s = check_device(h);
    if (s != BDECON_OK) return s;
    const int old = h->lean;
    const std::vector<Group> old_groups = h->groups;
    h->lean = mode;
    for (auto& g : h->groups) g.user_lean = -2;
    s = make_plan(h);
    if (s != BDECON_OK) {
        const std::string m = h->err;
        h->lean = old;
        h->groups = old_groups;
        make_plan(h);
        h->err = m;
    }
    return s;
}

bdecon_status bdecon_get_lean(bdecon_handle* h, int32_t p, int32_t* lean)
{
    if (!h || !lean) return fail(h, BDECON_ERR_INVALID, "bad arguments");
    if (p < 0 || p >= (int)h->probs.size()) return fail(h, BDECON_ERR_INVALID, "problem index %d", p);
    *lean = h->groups[h->prob_group[p]].lean ? 1 : 0;
    return BDECON_OK;
}

namespace {

// One autotuner trial: a segment of len sweeps in the current plan, timed
// per launch group.  Returns the per-group milliseconds (or an error).
bdecon_status tune_trial(bdecon_handle* h, int len, std::vector<double>& ms)
{
    const size_t ng = h->groups.size();
    std::vector<cudaEvent_t> ev(ng + 1);
    for (auto& e : ev) CK(h, cudaEventCreate(&e));
    LaunchSet ls;
    own_launch_set(h, ls);
    bdecon_status s = run_segment(ls, len, h->st, h, ev.data());
    if (s == BDECON_OK) s = check_device(h);
    ms.assign(ng, 0.0);
    if (s == BDECON_OK)
        for (size_t g = 0; g < ng; ++g) {
            float t = 0;
            cudaEventElapsedTime(&t, ev[g], ev[g + 1]);
            ms[g] = t;
        }
    for (auto& e : ev) cudaEventDestroy(e);
    return s;
}

}  // namespace

bdecon_status bdecon_autotune(bdecon_handle* h, int32_t trial_sweeps, int32_t* one_launch, double* ms_per_sweep)
{
    if (!h) return fail(nullptr, BDECON_ERR_INVALID, "handle is NULL");
    if (h->failed) return fail(h, BDECON_ERR_STATE, "handle failed earlier: %s", h->err.c_str());
    if (trial_sweeps < 1 || trial_sweeps > kMaxSlots) return fail(h, BDECON_ERR_INVALID, "trial_sweeps must be 1..%d", kMaxSlots);
    if (h->sweeps + trial_sweeps > h->max_sweeps)
        return fail(h, BDECON_ERR_INVALID, "trace capacity %d too small for %d trial sweeps after %lld", h->max_sweeps,
                    trial_sweeps, (long long)h->sweeps);
    bdecon_status s = check_device(h);
    if (s != BDECON_OK) return s;
    // snapshot: the whole workspace on the device, the counters on the host
    char* snap = nullptr;
    if (cudaMalloc(&snap, h->arena_bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, BDECON_ERR_NOMEM, "autotune needs a %zu-byte copy of the workspace", h->arena_bytes);
    }
    CK(h, cudaMemcpyAsync(snap, h->arena, h->arena_bytes, cudaMemcpyDeviceToDevice, h->st));
    const int64_t sweeps0 = h->sweeps;
    std::vector<int64_t> nsum0;
    for (const auto& ph : h->probs) nsum0.push_back(ph.n_sum);
    auto restore = [&]() -> bdecon_status {
        CK(h, cudaMemcpyAsync(h->arena, snap, h->arena_bytes, cudaMemcpyDeviceToDevice, h->st));
        CK(h, cudaStreamSynchronize(h->st));
        h->sweeps = sweeps0;
        for (size_t k = 0; k < h->probs.size(); ++k) h->probs[k].n_sum = nsum0[k];
        return BDECON_OK;
    };
    const int len = std::min<int>(trial_sweeps, segment_len(h, trial_sweeps));
    for (auto& ph : h->probs) ph.user_plan = false;
    static const int kMult[3] = {1, 2, 4};
    // (a) one launch per (L, S, team): each group's warps and residency tuned on its own
    h->one_launch = false;
    form_groups(h);
    std::vector<TuneChoice> best(h->groups.size());
    bool any_stage = false;   // window staging is a candidate only where some problem allows it
    for (const auto& ph : h->probs) any_stage = any_stage || ph.stage_ok;
    // (staged shapes are tried with the team's own warps only: their buffers
    // already limit the blocks per SM)
    // (the lean form is tried where it applies: float, unstaged)
    const int n_lean = h->precision == BDECON_FP32 ? 2 : 1;
    for (int st = 0; st <= (any_stage ? 1 : 0) && s == BDECON_OK; ++st)
        for (int ln = 0; ln < (st ? 1 : n_lean) && s == BDECON_OK; ++ln)
            for (int streamed = 0; streamed <= 1 && s == BDECON_OK; ++streamed)
                for (int mi = 0; mi < (st ? 1 : 3) && s == BDECON_OK; ++mi) {
                    bool any = false;
                    for (auto& g : h->groups) {
                        const int tw = g.team / 32, w = std::min(8, tw * kMult[mi]);
                        any = any || (mi == 0 || w != std::min(8, tw * kMult[mi - 1]));
                        g.warps = w;
                        g.user_warps = true;
                        g.streamed = streamed != 0;
                        g.no_stage = st == 0;
                        g.user_stage = true;
                        g.user_lean = ln;
                    }
                    if (!any) continue;
                    if (make_plan(h) != BDECON_OK) continue;   // no co-resident plan of this shape
                    if (ln == 1) {   // a lean trial only where some group runs the lean form
                        bool some = false;
                        for (const auto& g : h->groups) some = some || g.lean;
                        if (!some) continue;
                    }
                    std::vector<double> ms;
                    s = tune_trial(h, len, ms);
                    if (s == BDECON_OK) s = restore();
                    for (size_t g = 0; g < ms.size() && s == BDECON_OK; ++g)
                        if (ms[g] < best[g].ms)
                            best[g] = {h->groups[g].warps, streamed != 0, h->groups[g].stage == 1, ms[g], h->groups[g].lean};
                }
    double t_groups = 0;
    for (const auto& b : best) t_groups += b.ms;
    // (b) one launch over every problem
    TuneChoice one;
    if (s == BDECON_OK && h->probs.size() > 1) {
        h->one_launch = true;
        form_groups(h);
        Group& g = h->groups[0];
        bool behind = false;   // the first shapes are far slower than per-group launches: stop trying
        for (int st = 0; st <= (any_stage ? 1 : 0) && s == BDECON_OK && !behind; ++st)
            for (int streamed = 0; streamed <= 1 && s == BDECON_OK && !behind; ++streamed)
                for (int mi = 0; mi < (st ? 1 : 3) && s == BDECON_OK && !behind; ++mi) {
                    const int w = std::min(8, (g.team / 32) * kMult[mi]);
                    if (mi > 0 && w == std::min(8, (g.team / 32) * kMult[mi - 1])) continue;
                    g.warps = w;
                    g.user_warps = true;
                    g.streamed = streamed != 0;
                    g.no_stage = st == 0;
                    g.user_stage = true;
                    if (make_plan(h) != BDECON_OK) continue;
                    std::vector<double> ms;
                    s = tune_trial(h, len, ms);
                    if (s == BDECON_OK) s = restore();
                    if (s == BDECON_OK && ms[0] < one.ms) one = {w, streamed != 0, g.stage == 1, ms[0], g.lean};
                    behind = s == BDECON_OK && one.ms > 1.5 * t_groups;
                }
    }
    // apply the fastest
    if (s == BDECON_OK) {
        h->one_launch = one.ms < t_groups;
        form_groups(h);
        if (h->one_launch) {
            h->groups[0].warps = one.warps;
            h->groups[0].user_warps = true;
            h->groups[0].streamed = one.streamed;
            h->groups[0].no_stage = !one.staged;
            h->groups[0].user_stage = true;
            h->groups[0].user_lean = one.lean ? 1 : 0;
        } else {
            for (size_t g = 0; g < h->groups.size(); ++g) {
                h->groups[g].warps = best[g].warps;
                h->groups[g].user_warps = true;
                h->groups[g].streamed = best[g].streamed;
                h->groups[g].no_stage = !best[g].staged;
                h->groups[g].user_stage = true;
                h->groups[g].user_lean = best[g].lean ? 1 : 0;
            }
        }
        s = make_plan(h);
        if (one_launch) *one_launch = h->one_launch ? 1 : 0;
        if (ms_per_sweep) *ms_per_sweep = (h->one_launch ? one.ms : t_groups) / len;
        if (s == BDECON_OK) {
            TuneEntry e;
            e.one_launch = h->one_launch;
            for (const auto& g : h->groups) e.groups.push_back({g.warps, g.streamed, g.stage == 1, 0.0, g.lean});
            std::lock_guard<std::mutex> lock(g_tune_mu);
            if (g_tune_cache_on) g_tune_cache[tune_key(h)] = e;
        }
    }
    if (s != BDECON_OK) {
        const std::string m = h->err;
        restore();
        h->one_launch = false;
        form_groups(h);
        make_plan(h);
        h->err = m;
    }
    cudaFree(snap);
    return s;
}

bdecon_status bdecon_set_tuning_cache(int32_t enable)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache.clear();
    g_tune_cache_on = enable != 0;
    return BDECON_OK;
}

bdecon_status bdecon_get_plan(bdecon_handle* h, int32_t p, int32_t* blocks, int32_t* warps, int32_t* tile_i,
                              int32_t* tile_j)
{
    if (!h) return fail(nullptr, BDECON_ERR_INVALID, "handle is NULL");
    if (p < 0 || p >= (int)h->probs.size()) return fail(h, BDECON_ERR_INVALID, "problem index %d", p);
    const Group& g = h->groups[h->prob_group[p]];
    if (blocks) *blocks = g.grid;
    if (warps) *warps = g.warps;
    if (tile_i) *tile_i = h->probs[p].tpi;
    if (tile_j) *tile_j = h->probs[p].tpj;
    return BDECON_OK;
}

bdecon_status bdecon_launch_count(const bdecon_handle* h, int64_t* launches)
{
    if (!h || !launches) return fail(nullptr, BDECON_ERR_INVALID, "bad arguments");
    *launches = h->launches;
    return BDECON_OK;
}

bdecon_status bdecon_set_fault(bdecon_handle* h, int32_t silent_block, int64_t wait_ns)
{
    if (!h) return fail(nullptr, BDECON_ERR_INVALID, "handle is NULL");
    if (silent_block >= h->groups[0].grid) return fail(h, BDECON_ERR_INVALID, "block %d out of range", silent_block);
    if (wait_ns < 1000000 || wait_ns > 60000000000ll) return fail(h, BDECON_ERR_INVALID, "wait limit out of range");
    h->silent_block = silent_block < 0 ? -1 : silent_block;
    h->wait_ns = (unsigned long long)wait_ns;
    drop_graphs(h);   // captured launches carry the old values
    return BDECON_OK;
}

bdecon_status bdecon_set_timing(bdecon_handle* h, int32_t enable)
{
    if (!h) return fail(nullptr, BDECON_ERR_INVALID, "handle is NULL");
    h->timing = enable != 0;
    return BDECON_OK;
}

bdecon_status bdecon_sweep_kernel_time(bdecon_handle* h, double* ms, int64_t* launches)
{
    if (!h || !ms || !launches) return fail(h, BDECON_ERR_INVALID, "bad arguments");
    CK(h, cudaStreamSynchronize(h->st));
    double tot = 0.0;
    for (size_t k = 0; k + 1 < h->ev_used; k += 2) {
        float t = 0.f;
        CK(h, cudaEventElapsedTime(&t, h->ev_pool[k], h->ev_pool[k + 1]));
        tot += t;
    }
    *ms = tot;
    *launches = (int64_t)(h->ev_used / 2);
    h->ev_used = 0;
    return BDECON_OK;
}

}  // extern "C"

// ================================================================ serving
// Continuous batching: a worker thread admits queued jobs when a slot and
// device memory are free, sweeps every running job in shared cooperative
// launches (one per (L, S, team) across jobs, or one in all) per segment of
// at most segment_sweeps sweeps, and between segments retires finished jobs (their
// posterior mean is kept for polling) and admits new ones.  A job's chains
// keep their own sweep counter, refresh schedule and random stream, so its
// result does not depend on what else runs with it.
namespace {

struct SrvJob {
    int64_t id = 0;
    std::vector<float> image, gain, offset, var;
    std::vector<double> psf;
    bdecon_problem p{};
    int sweeps = 0, remaining = 0;
    int state = BDECON_JOB_QUEUED;
    double t_submit = 0, t_start = 0, t_done = 0;
    size_t mem = 0;
    bdecon_handle* h = nullptr;
    std::vector<double> mean;
    std::string err;
};

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct bdecon_server {
    bdecon_server_config cfg{};
    cudaStream_t st = nullptr;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    std::deque<int64_t> queue;
    std::map<int64_t, SrvJob*> jobs;
    std::vector<SrvJob*> active;        // worker-thread only
    std::vector<int64_t> job_cost;      // per running job: class steps x rounds x window pixels per sweep
    size_t mem_used = 0;
    int64_t next_id = 1;
    int64_t segments = 0;
    char* d_tab = nullptr;              // device tables of the shared launches
    size_t tab_cap = 0;
    bdecon_handle shell;                // error flag, precision, launch counter of the shared launches
    std::string err;
};

namespace {

bool srv_tables(bdecon_server* S, size_t bytes)
{
    if (bytes <= S->tab_cap) return true;
    if (S->d_tab) cudaFree(S->d_tab);
    S->d_tab = nullptr;
    S->tab_cap = 0;
    const size_t cap = std::max(bytes, (size_t)1 << 16);
    if (cudaMalloc(&S->d_tab, cap) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    S->tab_cap = cap;
    return true;
}

// Build the shared launch over the running jobs: a combined image table,
// one group per (L, S, team), chain copies in group order.
bool srv_build(bdecon_server* S, LaunchSet& ls, std::vector<Image>& imgs)
{
    ls = LaunchSet();
    imgs.clear();
    struct Entry { int hi, pk, img; };
    std::vector<Entry> ent;
    for (size_t hi = 0; hi < S->active.size(); ++hi) {
        bdecon_handle* h = S->active[hi]->h;
        ls.hs.push_back(h);
        for (size_t k = 0; k < h->probs.size(); ++k) {
            ent.push_back({(int)hi, (int)k, (int)imgs.size()});
            imgs.push_back(h->imgs[k]);
        }
    }
    // One launch per (L, S, team) across jobs, or one launch over every
    // running job (the kernel reads each block's problem from its chain).
    std::vector<std::vector<int>> groups;   // indices into ent
    for (size_t e = 0; e < ent.size(); ++e) {
        const bdecon_handle* h = ls.hs[ent[e].hi];
        const ProbHost& ph = h->probs[ent[e].pk];
        const int team = h->imgs[ent[e].pk].team;
        const int aug = ph.p.flags & BDECON_FLAG_AUGMENTED;
        const bool fine = ph.f > 1;
        int gi = -1;
        for (size_t q = 0; q < groups.size() && gi < 0; ++q) {
            const Entry& f = ent[groups[q][0]];
            const bdecon_handle* h2 = ls.hs[f.hi];
            const ProbHost& ph2 = h2->probs[f.pk];
            if ((ph2.p.flags & BDECON_FLAG_AUGMENTED) == aug && (ph2.f > 1) == fine &&
                (S->cfg.one_launch || (ph2.L == ph.L && ph2.S == ph.S && h2->imgs[f.pk].team == team)))
                gi = (int)q;
        }
        if (gi < 0) {
            groups.emplace_back();
            gi = (int)groups.size() - 1;
        }
        groups[gi].push_back((int)e);
    }
    // chain copies (img remapped), planned per group, laid out in group order
    std::vector<Chain> all;
    std::vector<int> all_owner, first(ent.size());
    for (size_t e = 0; e < ent.size(); ++e) {
        const bdecon_handle* h = ls.hs[ent[e].hi];
        const ProbHost& ph = h->probs[ent[e].pk];
        first[e] = (int)all.size();
        for (int c = 0; c < ph.p.n_chains; ++c) {
            Chain ch = h->chains[ph.chain0 + c];
            ch.img = ent[e].img;
            all.push_back(ch);
            all_owner.push_back(ent[e].hi);
        }
    }
    for (auto& gidx : groups) {
        Group g;
        g.aug = (ls.hs[ent[gidx[0]].hi]->probs[ent[gidx[0]].pk].p.flags & BDECON_FLAG_AUGMENTED) != 0;
        g.fine = ls.hs[ent[gidx[0]].hi]->probs[ent[gidx[0]].pk].f > 1;
        std::vector<PlanItem> items(gidx.size());
        std::vector<PlanItem*> ptrs;
        for (size_t q = 0; q < gidx.size(); ++q) {
            const Entry& e = ent[gidx[q]];
            const bdecon_handle* h = ls.hs[e.hi];
            PlanItem& it = items[q];
            it.ph = &h->probs[e.pk];
            it.team = h->imgs[e.pk].team;
            for (int c = 0; c < it.ph->p.n_chains; ++c) it.chains.push_back(&all[first[gidx[q]] + c]);
            ptrs.push_back(&it);
        }
        std::string err;
        if (!plan_items(S->shell.precision, S->shell.sms, ptrs, g, err)) {
            S->err = err;
            return false;
        }
        g.chain_off = (int)ls.gch.size();
        for (size_t q = 0; q < gidx.size(); ++q) {
            const Entry& e = ent[gidx[q]];
            for (int c = 0; c < ls.hs[e.hi]->probs[e.pk].p.n_chains; ++c) {
                ls.gch.push_back(all[first[gidx[q]] + c]);
                ls.owner.push_back(all_owner[first[gidx[q]] + c]);
            }
        }
        g.n_chains = (int)ls.gch.size() - g.chain_off;
        ls.groups.push_back(g);
    }
    // per job: the serial work of one sweep of its blocks
    // (class steps x patch rounds per team x window pixels), which sets its
    // sweeps per segment
    S->job_cost.assign(ls.hs.size(), 1);
    for (size_t gi = 0; gi < ls.groups.size(); ++gi) {
        const Group& g = ls.groups[gi];
        for (int k = g.chain_off; k < g.chain_off + g.n_chains; ++k) {
            const Chain& ch = ls.gch[k];
            const Image& im = imgs[ch.img];
            const int n_sub = std::max(1, g.threads / im.team);
            const int rounds = (ch.tpi * ch.tpj + n_sub - 1) / n_sub;
            S->job_cost[ls.owner[k]] = (int64_t)im.S * im.S * rounds * im.L * im.L;
        }
    }
    const size_t bi = sizeof(Image) * imgs.size(), bc = sizeof(Chain) * ls.gch.size();
    if (!srv_tables(S, align_up(bi, 256) + bc + 256)) {
        S->err = "cudaMalloc of the launch tables failed";
        return false;
    }
    if (cudaMemcpyAsync(S->d_tab, imgs.data(), bi, cudaMemcpyHostToDevice, S->st) != cudaSuccess) {
        S->err = "launch table upload failed";
        return false;
    }
    ls.d_imgs = (const Image*)S->d_tab;
    ls.d_gch = (Chain*)(S->d_tab + align_up(bi, 256));
    return true;
}

void srv_finish(bdecon_server* S, SrvJob* j, int state, std::string err)   // err by value: it may live in j->h
{
    if (j->h) {
        bdecon_destroy(j->h);
        j->h = nullptr;
    }
    std::lock_guard<std::mutex> lock(S->mu);
    S->mem_used -= j->mem;
    j->state = state;
    j->err = std::move(err);
    j->t_done = now_s();
    S->cv.notify_all();
}

void srv_loop(bdecon_server* S)
{
    cudaSetDevice(S->cfg.device);
    LaunchSet ls;
    std::vector<Image> imgs;
    bool dirty = true;
    for (;;) {
        std::vector<SrvJob*> admit;
        {
            std::unique_lock<std::mutex> lock(S->mu);
            if (S->active.empty() && S->queue.empty() && !S->stop)
                S->cv.wait_for(lock, std::chrono::milliseconds(20));
            if (S->stop) break;
            while (!S->queue.empty() && (int)(S->active.size() + admit.size()) < S->cfg.max_jobs) {
                SrvJob* j = S->jobs[S->queue.front()];
                if (S->mem_used + j->mem > S->cfg.mem_budget) break;   // wait for memory to free up
                S->queue.pop_front();
                S->mem_used += j->mem;
                admit.push_back(j);
            }
        }
        for (SrvJob* j : admit) {
            bdecon_status st = bdecon_create(&j->p, S->st, &j->h);
            if (st != BDECON_OK) {
                j->h = nullptr;
                srv_finish(S, j, BDECON_JOB_FAILED, bdecon_last_error(nullptr));
                continue;
            }
            {
                std::lock_guard<std::mutex> lock(S->mu);
                j->state = BDECON_JOB_RUNNING;
                j->t_start = now_s();
            }
            S->active.push_back(j);
            dirty = true;
        }
        if (S->active.empty()) continue;
        if (dirty) {
            if (!srv_build(S, ls, imgs)) {
                for (SrvJob* j : S->active) srv_finish(S, j, BDECON_JOB_FAILED, S->err);
                S->active.clear();
                continue;
            }
            dirty = false;
        }
        // sweeps per job in this segment: the job with the costliest sweep
        // takes segment_sweeps, jobs with cheaper sweeps proportionally more
        // (capped by the slot count, their next refresh and what they have
        // left), so light jobs finish early instead of with the heaviest
        int64_t cmax = 1;
        for (size_t hi = 0; hi < S->active.size(); ++hi) cmax = std::max(cmax, S->job_cost[hi]);
        std::vector<int> lens(S->active.size());
        int len = 1;
        for (size_t hi = 0; hi < S->active.size(); ++hi) {
            const int64_t want = (int64_t)S->cfg.segment_sweeps * cmax / S->job_cost[hi];
            lens[hi] = segment_len(S->active[hi]->h, (int)std::min<int64_t>({want, (int64_t)kMaxSlots,
                                                                             (int64_t)S->active[hi]->remaining}));
            len = std::max(len, lens[hi]);
        }
        for (size_t k = 0; k < ls.gch.size(); ++k) ls.gch[k].n_sweeps = lens[ls.owner[k]];
        bdecon_status st = BDECON_OK;
        if (cudaMemcpyAsync(ls.d_gch, ls.gch.data(), sizeof(Chain) * ls.gch.size(), cudaMemcpyHostToDevice, S->st) !=
            cudaSuccess) {
            cudaGetLastError();
            st = fail(&S->shell, BDECON_ERR_CUDA, "launch table upload failed");
        }
        if (st == BDECON_OK) st = run_segment(ls, len, S->st, &S->shell, nullptr, lens.data());
        if (st == BDECON_OK) st = check_device(&S->shell);
        if (st != BDECON_OK) {
            const std::string m = S->shell.err;
            for (SrvJob* j : S->active) srv_finish(S, j, BDECON_JOB_FAILED, m);
            S->active.clear();
            cudaMemsetAsync(S->shell.d_err, 0, 64, S->st);   // flags and the first-event record
            S->shell.failed = false;
            dirty = true;
            continue;
        }
        {
            std::lock_guard<std::mutex> lock(S->mu);
            ++S->segments;
        }
        std::vector<SrvJob*> keep;
        for (size_t hi = 0; hi < S->active.size(); ++hi) {
            SrvJob* j = S->active[hi];
            j->remaining -= lens[hi];
            if (j->remaining > 0) {
                keep.push_back(j);
                continue;
            }
            const ProbHost& ph = j->h->probs[0];
            j->mean.assign((size_t)ph.Ho * ph.Wo, 0.0);
            if (bdecon_posterior_mean(j->h, 0, j->mean.data(), 0) != BDECON_OK) {
                srv_finish(S, j, BDECON_JOB_FAILED, j->h->err);
            } else {
                srv_finish(S, j, BDECON_JOB_DONE, "");
            }
            dirty = true;
        }
        S->active.swap(keep);
    }
    for (SrvJob* j : S->active) srv_finish(S, j, BDECON_JOB_FAILED, "server stopped");
    S->active.clear();
}

}  // namespace

extern "C" {

bdecon_status bdecon_server_start(const bdecon_server_config* cfg, bdecon_server** out)
{
    if (!cfg || !out) return fail(nullptr, BDECON_ERR_INVALID, "bad arguments");
    *out = nullptr;
    if (cfg->max_jobs < 1 || cfg->segment_sweeps < 1 || cfg->segment_sweeps > kMaxSlots || cfg->mem_budget == 0 ||
        (cfg->precision != BDECON_FP32 && cfg->precision != BDECON_FP64))
        return fail(nullptr, BDECON_ERR_INVALID, "server config out of range");
    bdecon_server* S = new bdecon_server();
    S->cfg = *cfg;
    if (cudaSetDevice(cfg->device) != cudaSuccess || cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking) != cudaSuccess) {
        delete S;
        return fail(nullptr, BDECON_ERR_CUDA, "cannot use device %d", cfg->device);
    }
    S->shell.precision = cfg->precision;
    S->shell.st = S->st;
    cudaDeviceGetAttribute(&S->shell.sms, cudaDevAttrMultiProcessorCount, cfg->device);
    if (cudaMalloc(&S->shell.d_err, 256) != cudaSuccess || cudaMemset(S->shell.d_err, 0, 256) != cudaSuccess) {
        cudaStreamDestroy(S->st);
        delete S;
        return fail(nullptr, BDECON_ERR_NOMEM, "server error flag");
    }
    S->worker = std::thread(srv_loop, S);
    *out = S;
    return BDECON_OK;
}

bdecon_status bdecon_server_submit(bdecon_server* S, const bdecon_problem* p, int32_t sweeps, int64_t* job_id)
{
    if (!S || !p || !job_id) return fail(nullptr, BDECON_ERR_INVALID, "bad arguments");
    if (sweeps < 1) return fail(nullptr, BDECON_ERR_INVALID, "sweeps must be >= 1");
    if (sweeps <= p->burn_in)
        return fail(nullptr, BDECON_ERR_INVALID, "sweeps (%d) must exceed burn_in (%d): the job returns a posterior mean",
                    sweeps, p->burn_in);
    if (p->precision != S->cfg.precision) return fail(nullptr, BDECON_ERR_INVALID, "job precision differs from the server's");
    bdecon_status st = validate(*p, 0);
    if (st != BDECON_OK) return st;
    SrvJob* j = new SrvJob();
    const size_t n = (size_t)p->H * p->W;
    j->image.assign(p->image, p->image + n);
    if (p->gain_map) j->gain.assign(p->gain_map, p->gain_map + n);
    if (p->offset_map) j->offset.assign(p->offset_map, p->offset_map + n);
    if (p->var_map) j->var.assign(p->var_map, p->var_map + n);
    j->psf.assign(p->psf, p->psf + (size_t)p->L * p->L);
    j->p = *p;
    j->p.image = j->image.data();
    j->p.gain_map = p->gain_map ? j->gain.data() : nullptr;
    j->p.offset_map = p->offset_map ? j->offset.data() : nullptr;
    j->p.var_map = p->var_map ? j->var.data() : nullptr;
    j->p.psf = j->psf.data();
    j->p.max_sweeps = sweeps;
    j->p.flags = p->flags & BDECON_FLAG_AUGMENTED;
    j->sweeps = j->remaining = sweeps;
    size_t bytes = 0;
    st = bdecon_workspace_size(&j->p, 1, &bytes);
    if (st != BDECON_OK) {
        delete j;
        return st;
    }
    j->mem = bytes;
    j->t_submit = now_s();
    std::lock_guard<std::mutex> lock(S->mu);
    j->id = S->next_id++;
    S->jobs[j->id] = j;
    if (j->mem > S->cfg.mem_budget) {
        j->state = BDECON_JOB_FAILED;
        j->err = "job needs more device memory than the server budget";
        j->t_done = j->t_submit;
    } else {
        S->queue.push_back(j->id);
    }
    *job_id = j->id;
    S->cv.notify_all();
    return BDECON_OK;
}

bdecon_status bdecon_server_poll(bdecon_server* S, int64_t id, int32_t* state, double* times, double* mean, size_t cap)
{
    if (!S || !state) return fail(nullptr, BDECON_ERR_INVALID, "bad arguments");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->jobs.find(id);
    if (it == S->jobs.end()) return fail(nullptr, BDECON_ERR_INVALID, "unknown job %lld", (long long)id);
    SrvJob* j = it->second;
    *state = j->state;
    if (times) {
        times[0] = j->t_submit;
        times[1] = j->t_start;
        times[2] = j->t_done;
    }
    if (j->state == BDECON_JOB_FAILED) return fail(nullptr, BDECON_ERR_STATE, "job failed: %s", j->err.c_str());
    if (mean && j->state == BDECON_JOB_DONE) {
        if (cap < j->mean.size()) return fail(nullptr, BDECON_ERR_INVALID, "output capacity %zu < %zu", cap, j->mean.size());
        std::memcpy(mean, j->mean.data(), j->mean.size() * sizeof(double));
    }
    return BDECON_OK;
}

bdecon_status bdecon_server_wait(bdecon_server* S, int64_t id, double timeout_s, int32_t* state)
{
    if (!S || !state) return fail(nullptr, BDECON_ERR_INVALID, "bad arguments");
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->jobs.find(id);
    if (it == S->jobs.end()) return fail(nullptr, BDECON_ERR_INVALID, "unknown job %lld", (long long)id);
    SrvJob* j = it->second;
    S->cv.wait_for(lock, std::chrono::duration<double>(timeout_s),
                   [&] { return j->state == BDECON_JOB_DONE || j->state == BDECON_JOB_FAILED; });
    *state = j->state;
    return BDECON_OK;
}

bdecon_status bdecon_server_stats(bdecon_server* S, int64_t* queued, int64_t* running, int64_t* done, size_t* mem_used,
                                  int64_t* segments)
{
    if (!S) return fail(nullptr, BDECON_ERR_INVALID, "server is NULL");
    std::lock_guard<std::mutex> lock(S->mu);
    int64_t q = 0, r = 0, d = 0;
    for (auto& kv : S->jobs) {
        q += kv.second->state == BDECON_JOB_QUEUED;
        r += kv.second->state == BDECON_JOB_RUNNING;
        d += kv.second->state == BDECON_JOB_DONE;
    }
    if (queued) *queued = q;
    if (running) *running = r;
    if (done) *done = d;
    if (mem_used) *mem_used = S->mem_used;
    if (segments) *segments = S->segments;
    return BDECON_OK;
}

bdecon_status bdecon_server_stop(bdecon_server* S)
{
    if (!S) return fail(nullptr, BDECON_ERR_INVALID, "server is NULL");
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
        for (int64_t id : S->queue) {
            S->jobs[id]->state = BDECON_JOB_FAILED;
            S->jobs[id]->err = "server stopped";
        }
        S->queue.clear();
        S->cv.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    cudaStreamSynchronize(S->st);
    for (auto& kv : S->jobs) delete kv.second;
    if (S->d_tab) cudaFree(S->d_tab);
    if (S->shell.d_err) cudaFree(S->shell.d_err);
    cudaStreamDestroy(S->st);
    delete S;
    return BDECON_OK;
}

}  // extern "C"
