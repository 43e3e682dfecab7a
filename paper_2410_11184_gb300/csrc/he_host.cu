// Host orchestration of the RNS-CKKS hot path and the C ABI declared in include/he_gb300.h.
//
// Ciphertext batches live on the device as [n_ct][2][level+1][N] uint64 in NTT form.  The
// host only sequences kernel launches on the context stream and tracks levels and scales;
// all polynomial arithmetic runs in he_kernels.cu.  Scale bookkeeping, encoded constants and
// the order of operations follow the definitions written out in the comments below (the
// same definitions the CPU reference follows), so that results are bit-identical.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <set>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "he_kernels.cuh"
#include "../../include/he_gb300.h"

typedef unsigned __int128 u128;
typedef __int128 i128;

static const double HE_PI = 3.14159265358979323846;

// ------------------------------------------------------------------------- host arithmetic
static uint64_t h_mulmod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a * b) % q); }
static uint64_t h_pow(uint64_t a, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = h_mulmod(r, a, q);
        a = h_mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}
static uint64_t h_inv(uint64_t a, uint64_t q) { return h_pow(a % q, q - 2, q); }
static uint64_t h_shoup(uint64_t w, uint64_t q) { return (uint64_t)(((u128)w << 64) / q); }
// Montgomery form w 2^64 mod q of the constant factors that redc() sums over
static uint64_t h_mont(uint64_t w, uint64_t q) { return (uint64_t)(((u128)w << 64) % q); }
static uint64_t h_red128(i128 x, uint64_t q) {
    i128 r = x % (i128)q;
    if (r < 0) r += q;
    return (uint64_t)r;
}
static i128 h_round(double x) { return (i128)nearbyint(x); }
static int ilog2c(int x) { int r = 0; while ((1 << r) < x) r++; return r; }

// primitive 2N-th root of unity: the first g^((q-1)/2N) (g = 2, 3, ...) with N-th power -1
static uint64_t h_root(uint64_t q, int n) {
    uint64_t e = (q - 1) / (2 * (uint64_t)n);
    for (uint64_t g = 2; g < 1000000; g++) {
        uint64_t x = h_pow(g, e, q);
        if (h_pow(x, n, q) == q - 1) return x;
    }
    return 0;
}

// ------------------------------------------------------------------------- context
struct DCt;
using DPtr = std::shared_ptr<uint64_t>;

struct LtPlain {
    int a, b;          // giant index, baby index
    DPtr pt;           // [level+1][N] NTT
};
struct LtLevel {
    int hmin, g, E;
    std::vector<int> baby;           // baby steps b present
    std::vector<LtPlain> pts;
};

struct he_ctx {
    int logN = 0, N = 0, n0 = 0, nq = 0, np = 0, alpha = 0, h = 0, nm = 0;
    double sigma = 3.2;
    int log_scale = 40, user_top = 0, bootstrap = 0, stc_levels = 3, cts_levels = 3, bts_min = 3;
    double em_K = 0;
    int em_r = 0, em_deg = 0;
    std::vector<double> em_c;
    std::vector<uint64_t> mods;
    std::vector<ModC> modc;
    ModC *d_mods = nullptr;
    uint64_t *d_ninv = nullptr;
    // inverse-transform scale factors with a basis conversion's first factor folded in, per prime
    // index (N^{-1} [qhat_i^{-1}]_{q_i}, Shoup): ModUp per level [nq][nm][2] (qhat within the
    // limb's digit), ModDown [nm][2] (qhat within P), relinearise + rescale per level [nq][nm][2]
    // (qhat within {q_l} u P)
    uint64_t *d_ninv_up = nullptr, *d_ninv_down = nullptr, *d_ninv_rr = nullptr;
    ulonglong2 *d_tw2 = nullptr;   // per modulus: N (w, w') forward twiddle pairs, then N inverse pairs
    std::vector<std::vector<size_t>> cv_off;
    uint64_t *d_cv = nullptr;
    uint64_t *d_mdcv = nullptr, *d_pinv = nullptr, *d_qlinv = nullptr;
    int *d_pidx = nullptr;
    // relinearisation + rescale as one division by P q_l (per level l): conversion constants
    // from D = {q_l} u P (layout of the ModDown table, alpha + 1 sources), the sources' prime
    // indices, and per kept limb i: (P mod q_i, Shoup), ((P q_l)^{-1} mod q_i, Shoup)
    uint64_t *d_rrcv = nullptr, *d_rrpq = nullptr;
    int *d_rridx = nullptr;
    size_t rrcv_stride = 0;
    double2 *d_zeta = nullptr;
    int *d_rg = nullptr;
    std::vector<double2> zeta;
    std::vector<int> rg;
    uint64_t *d_cdt = nullptr;
    int cdt_len = 0;
    uint64_t *d_radix = nullptr, *d_radinv = nullptr;
    double *d_qd = nullptr;
    bool have_keys = false;
    uint64_t seed = 0;
    uint64_t *d_s = nullptr, *d_pk = nullptr;
    std::map<int, uint64_t *> keys;
    int ndig_top = 0;
    std::map<std::string, LtLevel> lt_cache;
    std::map<std::string, DPtr> pt_cache;   // Softmax masks, encoded once per (level, scale, stride)
    struct ProfRec {
        const char *fam;
        double bytes;
        cudaEvent_t a, b;
    };
    struct SmGraph {
        cudaGraphExec_t exec = nullptr;
        int level = 0;
        double scale = 0;
        long launches = 0;
        long cnt[5] = {0, 0, 0, 0, 0};
        std::vector<ProfRec> prof;   // timing events captured into the graph (profiling on)
        bool replayed = false;       // launched since the last he_profile_read/breakdown
    };
    std::vector<ProfRec> cap_prof;   // events recorded while capturing
    // graphs are captured and launched on a stream of their own (the context stream may be the
    // legacy default stream, which cannot be captured), ordered after / before the context
    // stream by events
    cudaStream_t gstream = nullptr;
    cudaEvent_t gev_in = nullptr, gev_out = nullptr;
    std::map<std::string, SmGraph> graphs;  // captured Softmax circuits (he_softmax_graph)
    // plans registered with he_softmax_register, by (n, M, method): deep copies whose arrays the
    // context owns (the he_softmax_plan points into the vectors of its own map node)
    struct PlanCopy {
        he_softmax_plan p;
        std::vector<double> exp_c, inv_c, a, b, gs, gl, expo, lam_max, b_max;
        std::vector<int> deg;
    };
    std::map<std::tuple<int, double, int>, PlanCopy> plans;
    bool capturing = false;
    uint64_t *noalloc_scratch = nullptr;   // device address of g_rescale_scratch on this device
    // launch-strategy choices of the autotuner (he_autotune): (operation, limbs, ciphertexts) ->
    // variant; tune_force[op] >= 0 overrides the table (tests); every variant gives the same words
    struct TuneRec {
        int choice;
        float ms[2];
    };
    std::map<std::tuple<int, int, int>, TuneRec> tune;
    int tune_force[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
    // CTA size of the transforms per direction (forward, inverse): the autotuner's choice at each
    // limb count of its ladder; a launch takes the choice of the largest ladder count <= its own
    std::vector<std::pair<int, int>> ntt_small[2];
    // one-pass transforms (N = 2^16, no fused neighbours) per direction: the autotuner's choice at
    // each limb count of its ladder, as for ntt_small (off until tuned)
    std::vector<std::pair<int, int>> ntt_1pass[2];
    cudaStream_t st = nullptr;
    // side streams for independent branches of a circuit (Branch), created on first use
    static const int NSIDE = 4;
    cudaStream_t side[NSIDE] = {};
    cudaEvent_t fork_ev[NSIDE] = {}, join_ev[NSIDE] = {};
    int branch_depth = 0;   // > 0 while a Branch is entered
    int next_side = 0;      // round-robin choice of the side stream for the next branch
    std::string err;
    long cnt[5] = {0, 0, 0, 0, 0};
    long launches = 0;
    int max_grid = 152 * 16;
    // live kernel timing: CUDA events around the launches of one kernel family
    std::string prof_name;   // a family name, or "all"
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev;
    std::vector<const char *> prof_fam;   // family of each recorded launch
    std::vector<const char *> prof_ph;    // circuit phase of each recorded launch
    std::vector<double> prof_b;           // its algorithmic bytes
    const char *phase = "other";          // circuit phase of the launches being issued (PhaseScope)
    size_t prof_used = 0;
    double prof_bytes = 0;
};

// Records events around one launch (or one copy) of kernel family `name` when that family,
// or "all", is the profiled one.  Every scope brackets exactly one launch, so the families'
// times add up to the stream's busy time.
struct ProfScope {
    he_ctx *c;
    bool on;
    size_t slot;
    bool cap = false;
    ProfScope(he_ctx *c_, const char *name, double bytes) : c(c_), on(match(c_->prof_name, name)) {
        if (!on) return;
        if (c->capturing) {
            // inside a graph capture: external event-record nodes, owned by the graph
            cap = true;
            he_ctx::ProfRec r{name, bytes, nullptr, nullptr};
            cudaEventCreate(&r.a);
            cudaEventCreate(&r.b);
            cudaEventRecordWithFlags(r.a, c->st, cudaEventRecordExternal);
            c->cap_prof.push_back(r);
            slot = c->cap_prof.size() - 1;
            return;
        }
        if (c->prof_used == c->prof_ev.size()) {
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            c->prof_ev.push_back({a, b});
            c->prof_fam.push_back(nullptr);
            c->prof_ph.push_back(nullptr);
            c->prof_b.push_back(0);
        }
        slot = c->prof_used++;
        c->prof_fam[slot] = name;
        c->prof_ph[slot] = c->phase;
        c->prof_b[slot] = bytes;
        c->prof_bytes += bytes;
        cudaEventRecord(c->prof_ev[slot].first, c->st);
    }
    // "all", the family itself, or a family prefix ("ntt" covers "ntt_modup", ...)
    static bool match(const std::string &want, const char *name) {
        if (want.empty()) return false;
        if (want == "all" || want == name) return true;
        size_t n = want.size();
        return strncmp(name, want.c_str(), n) == 0 && name[n] == '_';
    }
    ~ProfScope() {
        if (!on) return;
        if (cap) cudaEventRecordWithFlags(c->cap_prof[slot].b, c->st, cudaEventRecordExternal);
        else cudaEventRecord(c->prof_ev[slot].second, c->st);
    }
};

// Marks the launches issued in its lifetime as one phase of the Softmax circuit (main thread,
// auxiliary thread, bootstrapping): an NVTX range for profilers, and the phase recorded with
// every launch timed by ProfScope (he_profile_breakdown sums per phase).  Nested scopes take
// over and hand back.
struct PhaseScope {
    struct he_ctx *c;
    const char *prev;
    PhaseScope(struct he_ctx *c_, const char *name);
    ~PhaseScope();
};

struct HeErr {
    int code;
    std::string msg;
};

PhaseScope::PhaseScope(he_ctx *c_, const char *name) : c(c_), prev(c_->phase) {
    c->phase = name;
    nvtxRangePushA(name);
}
PhaseScope::~PhaseScope() {
    nvtxRangePop();
    c->phase = prev;
}

#define CK(call)                                                                                     \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) throw HeErr{HE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
    } while (0)
#define LAUNCH_CHECK()              \
    do {                            \
        c->launches++;              \
        CK(cudaGetLastError());     \
    } while (0)
#define REQUIRE(cond, code, msg)                                          \
    do {                                                                  \
        if (!(cond)) throw HeErr{code, msg};                              \
    } while (0)

// Stream-ordered device buffers.  A buffer is freed on the stream that is current when its last
// reference goes (c->st then), not on the one it was allocated on: inside a Branch that is the
// branch's stream, which follows every use of the buffer before the fork and in the branch;
// after the join it is the main stream, which follows the branch.  A buffer is never in use on
// two branches at once unless an outer scope holds it.
static DPtr dalloc(he_ctx *c, size_t words) {
    void *p = nullptr;
    if (words == 0) words = 1;
    cudaError_t e = cudaMallocAsync(&p, words * 8, c->st);
    if (e != cudaSuccess) throw HeErr{HE_ENOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e)};
    return DPtr((uint64_t *)p, [c](uint64_t *q) { cudaFreeAsync(q, c->st); });
}

// An independent branch of a circuit on side stream i.  Construction forks it from the work
// issued so far on the current (main) stream; between enter() and leave() the library issues on
// the side stream; join() (or the destructor) makes the main stream wait for the branch.  Several
// branches forked at the same point run concurrently with each other and with what the main
// stream does before the joins; inside a graph capture they become parallel branches of the graph.
struct Branch {
    he_ctx *c;
    cudaStream_t main;
    int i;
    bool joined = false, inside = false;
    // side stream i, or the next one round-robin with i < 0
    bool on;
    Branch(he_ctx *c_, int i_ = -1)
        : c(c_), main(c_->st), i(i_ >= 0 ? i_ : c_->next_side++ % he_ctx::NSIDE), on(c_->tune_force[HE_TUNE_BRANCHES] != 0) {
        if (!on) return;   // serial: everything stays on the context stream
        if (!c->side[i]) {
            CK(cudaStreamCreateWithFlags(&c->side[i], cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&c->fork_ev[i], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&c->join_ev[i], cudaEventDisableTiming));
        }
        CK(cudaEventRecord(c->fork_ev[i], main));
        CK(cudaStreamWaitEvent(c->side[i], c->fork_ev[i], 0));
    }
    void enter() {
        if (!on) return;
        c->st = c->side[i];
        c->branch_depth++;
        inside = true;
    }
    void leave() {
        if (!on || !inside) return;
        inside = false;
        c->branch_depth--;
        c->st = main;
    }
    void join() {
        leave();
        if (!on || joined) return;
        joined = true;
        cudaEventRecord(c->join_ev[i], c->side[i]);
        cudaStreamWaitEvent(main, c->join_ev[i], 0);
    }
    ~Branch() { join(); }
};

// a cache entry (encoded diagonals or masks) made inside a Branch may be read by another branch
// or the main stream: outside a graph capture, finish it before it is shared (first use only;
// captures run after an eager pass has filled the caches)
static void cache_entry_made(he_ctx *c) {
    if (c->branch_depth > 0 && !c->capturing) CK(cudaStreamSynchronize(c->st));
}

static dim3 grid_for(he_ctx *c, long total) {
    long b = (total + 255) / 256;
    return dim3((unsigned)std::max(1L, std::min(b, (long)c->max_grid)));
}

// ------------------------------------------------------------------------- launch strategies
// Bit-identical alternatives the autotuner chooses between, per (operation, limbs, ciphertexts):
//   HE_TUNE_MODUP     1: every digit of the ModUp converted in one launch and transformed in one
//                     more; 0: one conversion and two transforms per digit
//   HE_TUNE_ROT       1: the key switches of several hoisted rotations in one inner-product launch
//                     and one ModDown over all; 0: one key switch per rotation
//   HE_TUNE_LT_SMALL  1: one ModUp of every giant-step sum of a linear-transform level and one
//                     launch summing their inner products; 0: a ModUp per giant step
//   HE_TUNE_LT_ROWS   1: inner sums without shared-memory staging; 0: staged diagonal tiles
//   HE_TUNE_BRANCHES  1: independent branches of a circuit on side streams (Branch); 0: every
//                     launch on the context stream, in the same order as the host issues it
//   HE_TUNE_NTT_SMALL 1: the transform in CTAs of 64 threads (4 sub-transforms each); 0: 256
//                     threads.  Chosen per direction from a ladder of limb counts (ntt_small).
//   HE_TUNE_NTT_1PASS 1: a transform of N = 2^16 limbs without fused neighbours as one launch
//                     per limb cluster (16 CTAs, the passes' exchange in distributed shared
//                     memory); 0: the two register-blocked passes.  Per direction and limb count
//                     from a ladder (ntt_1pass); off until tuned.
//   HE_TUNE_FUSE_CONV 1: the basis conversions of ModUp and ModDown computed in the column pass
//                     of the forward transform that follows them (NttFuse kinds 4-6); 0: a
//                     conversion kernel writes the converted limbs, then the transform reads them
// Defaults (no table entry): 1 for batches of at most 4 ciphertexts (8 rows for LT_ROWS);
// branches on; separate conversions (the fused ones measured slower: their column-strided
// re-reads of the source limbs for every target limb leave the pass latency-bound).
static int tune_pick(he_ctx *c, int op, int L, int nct, int dflt) {
    if (c->tune_force[op] >= 0) return c->tune_force[op];
    auto it = c->tune.find(std::make_tuple(op, L, nct));
    return it == c->tune.end() ? dflt : it->second.choice;
}

// ------------------------------------------------------------------------- limb maps
static LimbMap qmap(int L) {
    LimbMap m;
    m.nper = L;
    for (int i = 0; i < L; i++) m.prime[i] = i;
    return m;
}
static LimbMap extmap(he_ctx *c, int L) {
    LimbMap m;
    m.nper = L + c->alpha;
    for (int i = 0; i < L; i++) m.prime[i] = i;
    for (int k = 0; k < c->alpha; k++) m.prime[L + k] = c->nq + k;
    return m;
}
static LimbMap pmap(he_ctx *c) {
    LimbMap m;
    m.nper = c->alpha;
    for (int k = 0; k < c->alpha; k++) m.prime[k] = c->nq + k;
    return m;
}
static LimbMap allmap(he_ctx *c) {
    LimbMap m;
    m.nper = c->nm;
    for (int i = 0; i < c->nm; i++) m.prime[i] = i;
    return m;
}
static LimbMap single(int p) {
    LimbMap m;
    m.nper = 1;
    m.prime[0] = p;
    return m;
}

// ------------------------------------------------------------------------- NTT launches
static const char *ntt_inv_family(const char *site) {
    static const char *const fwd[] = {"ntt", "ntt_modup", "ntt_moddown", "ntt_rescale", "ntt_modraise"};
    static const char *const inv[] = {"ntt_inv", "ntt_modup_inv", "ntt_moddown_inv", "ntt_rescale_inv",
                                      "ntt_modraise_inv"};
    for (int i = 0; i < 5; i++)
        if (!strcmp(site, fwd[i])) return inv[i];
    return "ntt_inv";
}

// NTT of `count` limbs in place, or out of place from src (limb l of polynomial i at
// src + i src_stride + l N) when src is given; register-blocked passes of 8 (N = 2^12) or 16
// (N = 2^16) coefficients per thread, the only ring sizes a context accepts.
// fuse: neighbours of a forward transform, see NttFuse
// ninv: the inverse transform's per-prime scale factors (default N^{-1}; a d_ninv_* table folds a
// basis conversion's first factor in)
static void ntt(he_ctx *c, uint64_t *base, int count, const LimbMap &map, long poly_stride, bool inverse,
                const char *site = "ntt", const uint64_t *src = nullptr, long src_stride = 0,
                const NttFuse *fuse = nullptr, const uint64_t *ninv = nullptr) {
    if (count <= 0) return;
    REQUIRE(!fuse || !inverse, HE_EINVAL, "fused transform: forward only");
    // timing family: the call site with the direction ("ntt_modup" forward, "ntt_modup_inv"
    // inverse); algorithmic bytes: the transform's read + write of every limb, 16 N per limb
    // (kind 7 leaves the digits' own limbs: ndc digits per group of ndc polynomials)
    long work = count;
    if (fuse && fuse->kind == 7) {
        long own = 0;
        for (int j = 0; j < fuse->ndc; j++) own += fuse->dds[j];
        work -= (long)count / ((long)map.nper * fuse->ndc) * own;
    }
    ProfScope ps(c, inverse ? ntt_inv_family(site) : site, 16.0 * work * c->N);
    c->launches++;
    if (c->logN == 16 && !fuse) {
        bool one = false;
        if (c->tune_force[HE_TUNE_NTT_1PASS] >= 0) {
            one = c->tune_force[HE_TUNE_NTT_1PASS] == 1;
        } else {
            for (const auto &e : c->ntt_1pass[inverse ? 1 : 0])   // ascending limb counts
                if (e.first <= count) one = e.second == 1;
        }
        if (one) {
            launch_ntt_1pass(inverse, count, base, map.nper, poly_stride, map, c->d_mods, c->d_tw2,
                             ninv ? ninv : c->d_ninv, c->logN, c->st, src, src_stride);
            LAUNCH_CHECK();
            return;
        }
    }
    bool small = false;
    if (c->tune_force[HE_TUNE_NTT_SMALL] >= 0) {
        small = c->tune_force[HE_TUNE_NTT_SMALL] == 1;
    } else {
        for (const auto &e : c->ntt_small[inverse ? 1 : 0])   // ascending limb counts
            if (e.first <= count) small = e.second == 1;
    }
    launch_ntt_rb(c->logN == 16 ? 4 : 3, inverse, count, base, map.nper, poly_stride, map, c->d_mods, c->d_tw2,
                  ninv ? ninv : c->d_ninv, c->logN, c->st, src, src_stride, fuse, small);
    LAUNCH_CHECK();
}

// ------------------------------------------------------------------------- ciphertexts
struct DCt {
    DPtr buf;              // owner (empty when viewing caller memory)
    uint64_t *d = nullptr;
    int level = 0;
    double scale = 1.0;
    int nct = 1;
    long cs(const he_ctx *c) const { return 2L * (level + 1) * c->N; }   // ciphertext stride
    long ps(const he_ctx *c) const { return (long)(level + 1) * c->N; }  // polynomial stride
};

static DCt ct_new(he_ctx *c, int level, int nct, double scale) {
    DCt x;
    x.level = level;
    x.nct = nct;
    x.scale = scale;
    x.buf = dalloc(c, (size_t)nct * 2 * (level + 1) * c->N);
    x.d = x.buf.get();
    return x;
}

// a caller's ciphertext batch; descriptors that could reach a kernel out of bounds are refused
static DCt ct_view(const he_ctx *c, const he_ct *h) {
    REQUIRE(h && h->data && h->n_ct >= 1 && h->level >= 0 && h->level < c->nq, HE_EINVAL,
            "ciphertext: data must be set, n_ct >= 1 and 0 <= level < n_q");
    DCt x;
    x.d = h->data;
    x.level = h->level;
    x.scale = h->scale;
    x.nct = h->n_ct;
    return x;
}

static DCt ct_copy(he_ctx *c, const DCt &a) {
    DCt y = ct_new(c, a.level, a.nct, a.scale);
    {
        ProfScope ps_(c, "copy", 0);
        CK(cudaMemcpyAsync(y.d, a.d, (size_t)a.nct * a.cs(c) * 8, cudaMemcpyDeviceToDevice, c->st));
    }
    return y;
}

// copy of a with only limbs 0..level (dropping limbs keeps value mod the smaller Q and scale)
static DCt ct_drop(he_ctx *c, const DCt &a, int level) {
    REQUIRE(level <= a.level && level >= 0, HE_ELEVEL, "drop: level");
    if (level == a.level) return ct_copy(c, a);
    DCt y = ct_new(c, level, a.nct, a.scale);
    {
        ProfScope ps_(c, "copy", 0);
        CK(cudaMemcpy2DAsync(y.d, (size_t)y.ps(c) * 8, a.d, (size_t)a.ps(c) * 8, (size_t)y.ps(c) * 8, 2 * a.nct,
                             cudaMemcpyDeviceToDevice, c->st));
    }
    return y;
}

// one ciphertext of a batch, as a view
static DCt ct_sub(const he_ctx *c, const DCt &a, int i) {
    DCt y;
    y.buf = a.buf;
    y.d = a.d + (long)i * a.cs(c);
    y.level = a.level;
    y.scale = a.scale;
    y.nct = 1;
    return y;
}

static bool scales_match(double a, double b) { return std::fabs(a - b) <= 1e-9 * std::fabs(a); }

static void ct_add_inplace(he_ctx *c, DCt &a, const DCt &b, bool sub = false) {
    REQUIRE(a.level == b.level && a.nct == b.nct, HE_EINVAL, "add: level/count mismatch");
    REQUIRE(scales_match(a.scale, b.scale), HE_EINVAL, "add: scale mismatch");
    int count = 2 * a.nct * (a.level + 1);
    LimbMap m = qmap(a.level + 1);
    long total = (long)count << c->logN;
    {
        ProfScope ps_(c, "elementwise", 0);
        klaunch(k_add, grid_for(c, total), 256, 0, c->st)(a.d, a.ps(c), a.d, a.ps(c), b.d, b.ps(c), count, a.level + 1, m,
                                                      c->d_mods, c->logN, sub ? 1 : 0);
    }
    LAUNCH_CHECK();
}

static Scal scal_of(he_ctx *c, i128 k, int L) {
    Scal s;
    for (int i = 0; i < L; i++) s.v[i] = h_red128(k, c->mods[i]);
    return s;
}

static void ct_mul_int(he_ctx *c, DCt &a, i128 k) {
    int L = a.level + 1, count = 2 * a.nct * L;
    Scal s = scal_of(c, k, L);
    {
        ProfScope ps_(c, "elementwise", 0);
        klaunch(k_mul_scalar, grid_for(c, (long)count << c->logN), 256, 0, c->st)(a.d, a.ps(c), a.d, a.ps(c), s, count, L,
                                                                              qmap(L), c->d_mods, c->logN);
    }
    LAUNCH_CHECK();
}

// adds the constant k (every slot, as a constant polynomial) to c0 of every ciphertext
static void ct_add_const(he_ctx *c, DCt &a, i128 k) {
    int L = a.level + 1, count = a.nct * L;
    Scal s = scal_of(c, k, L);
    {
        ProfScope ps_(c, "elementwise", 0);
        klaunch(k_add_scalar, grid_for(c, (long)count << c->logN), 256, 0, c->st)(a.d, a.cs(c), s, count, L, qmap(L),
                                                                              c->d_mods, c->logN);
    }
    LAUNCH_CHECK();
}

static void ct_mul_plain(he_ctx *c, DCt &a, const uint64_t *pt) {
    int L = a.level + 1, count = 2 * a.nct * L;
    {
        ProfScope ps_(c, "elementwise", 0);
        klaunch(k_mul, grid_for(c, (long)count << c->logN), 256, 0, c->st)(a.d, a.ps(c), a.d, a.ps(c), pt, 0, count, L, qmap(L),
                                                                       c->d_mods, c->logN, 0);
    }
    LAUNCH_CHECK();
}

// rescale: r = centred last limb; c_i <- (c_i - r) q_l^{-1}
static DCt rescale(he_ctx *c, const DCt &a) {
    int l = a.level, L = l + 1;
    REQUIRE(l >= 1, HE_ELEVEL, "rescale at level 0");
    int npoly = 2 * a.nct;
    DPtr last = dalloc(c, (size_t)npoly * c->N);
    ntt(c, last.get(), npoly, single(l), c->N, true, "ntt_rescale", a.d + (long)l * c->N, (long)L * c->N);
    DPtr tmp = dalloc(c, (size_t)npoly * l * c->N);
    // spread of the centred last limb and the final (x - t) q_l^{-1} fused into the transform
    DCt y = ct_new(c, l - 1, a.nct, a.scale / (double)c->mods[l]);
    NttFuse F{};
    F.kind = 2;
    F.x = a.d;
    F.out = y.d;
    F.cst = c->d_qlinv + (size_t)l * 2 * c->nq;
    F.last = last.get();
    F.ql = c->mods[l];
    ntt(c, tmp.get(), npoly * l, qmap(l), (long)l * c->N, false, "ntt_rescale", nullptr, 0, &F);
    c->cnt[3]++;
    return y;
}

// ------------------------------------------------------------------------- rescale, no allocation
// Scratch of he_rescale_noalloc: a file-scope device array, so that the call allocates nothing.
// It holds the centred last limbs and their spread over the remaining limbs:
// 2 n_ct (level + 1) N words at most (2 Mi words = 16 MiB).  Every device that loads this
// library reserves it until the process exits.
#define HE_NOALLOC_SCRATCH_WORDS (2u << 20)
static __device__ __align__(256) uint64_t g_rescale_scratch[HE_NOALLOC_SCRATCH_WORDS];

// the same steps as rescale(), with the scratch above and the caller's output buffer
static void rescale_noalloc(he_ctx *c, const DCt &a, uint64_t *out) {
    int l = a.level, L = l + 1, npoly = 2 * a.nct;
    uint64_t *last = c->noalloc_scratch, *tmp = last + (size_t)npoly * c->N;
    CK(cudaMemcpy2DAsync(last, (size_t)c->N * 8, a.d + (long)l * c->N, (size_t)L * c->N * 8, (size_t)c->N * 8, npoly,
                         cudaMemcpyDeviceToDevice, c->st));
    ntt(c, last, npoly, single(l), c->N, true);
    long tot = (long)npoly * l << c->logN;
    klaunch(k_rescale_spread, grid_for(c, tot), 256, 0, c->st)(tmp, last, npoly, l, qmap(l), c->d_mods, c->mods[l], c->logN);
    LAUNCH_CHECK();
    ntt(c, tmp, npoly * l, qmap(l), (long)l * c->N, false);
    klaunch(k_rescale_fin, grid_for(c, tot), 256, 0, c->st)(out, a.d, tmp, npoly, L, qmap(l), c->d_mods,
                                                        c->d_qlinv + (size_t)l * 2 * c->nq, c->logN);
    LAUNCH_CHECK();
    c->cnt[3]++;
}

// ------------------------------------------------------------------------- key switching
// ModUp of nct polynomials x (NTT form, L limbs, stride sx between polynomials):
// digits [nct][ndig][L + alpha][N] in NTT form.  The inverse transform multiplies limb i by
// N^{-1} [qhat_i^{-1}]_{q_i} (qhat within its digit), the conversion's first factor.
static DPtr ks_modup(he_ctx *c, const uint64_t *x, long sx, int nct, int L) {
    int al = c->alpha, nd = (L + al - 1) / al, nl = L + al;
    DPtr tmp = dalloc(c, (size_t)nct * L * c->N);
    ntt(c, tmp.get(), nct * L, qmap(L), (long)L * c->N, true, "ntt_modup", x, sx, nullptr,
        c->d_ninv_up + (size_t)(L - 1) * 2 * c->nm);
    DPtr dig = dalloc(c, (size_t)nct * nd * nl * c->N);
    LimbMap em = extmap(c, L);
    const bool all = tune_pick(c, HE_TUNE_MODUP, L, nct, nct <= 4);
    if (tune_pick(c, HE_TUNE_FUSE_CONV, L, nct, 0)) {
        // conversion in the column pass of the forward transform (NttFuse kind 4): every limb of
        // the extended basis outside the digit is converted and transformed in one pass pair,
        // the digit's own limbs are copied from x; all digits in one launch (all) or one per digit
        NttFuse F{};
        F.kind = 4;
        F.src = tmp.get();
        F.sstride = (long)L * c->N;
        F.cvw = c->d_cv + c->cv_off[L - 1][0];
        F.wstride = nl;
        F.xntt = x;
        F.sxn = sx;
        for (int j = 0; j < nd; j++) {
            F.dlo[j] = j * al;
            F.dds[j] = std::min(al, L - j * al);
            F.dcv[j] = (long)(c->cv_off[L - 1][j] - c->cv_off[L - 1][0]) + 2 * F.dds[j];
        }
        if (all) {
            F.ndc = nd;
            F.j0 = 0;
            ntt(c, dig.get(), nct * nd * nl, em, (long)nl * c->N, false, "ntt_modup", nullptr, 0, &F);
        } else {
            F.ndc = 1;
            for (int j = 0; j < nd; j++) {
                F.j0 = j;
                ntt(c, dig.get() + (long)j * nl * c->N, nct * nl, em, (long)nd * nl * c->N, false, "ntt_modup", nullptr,
                    0, &F);
            }
        }
        return dig;
    }
    if (all) {
        // small batches: every digit converted in one launch and transformed in one more (the
        // per-digit launches would each fill a fraction of the GPU); the digit's own limbs are
        // converted too, which reproduces them exactly
        ModUpDigits D{};
        for (int j = 0; j < nd; j++) {
            D.lo[j] = j * al;
            D.ds[j] = std::min(al, L - j * al);
            D.cvoff[j] = (long)c->cv_off[L - 1][j] - (long)c->cv_off[L - 1][0];
        }
        dim3 grid(grid_for(c, (long)nct << c->logN).x, nd);
        {
            ProfScope ps(c, "modup", 8.0 * c->N * ((double)nct * L + (double)nct * nd * nl));
            klaunch(k_modup_all, grid, 256, 0, c->st)(dig.get(), (long)nd * nl * c->N, tmp.get(), (long)L * c->N, nct, D, nl,
                                                 em, c->d_mods, c->d_cv + c->cv_off[L - 1][0], c->logN, x, sx);
        }
        LAUNCH_CHECK();
        // the digits' own limbs were copied in NTT form: the transform leaves them (kind 7)
        NttFuse F{};
        F.kind = 7;
        F.ndc = nd;
        F.j0 = 0;
        for (int j = 0; j < nd; j++) {
            F.dlo[j] = D.lo[j];
            F.dds[j] = D.ds[j];
        }
        ntt(c, dig.get(), nct * nd * nl, em, (long)nl * c->N, false, "ntt_modup", nullptr, 0, &F);
        return dig;
    }
    for (int j = 0; j < nd; j++) {
        int lo = j * al, ds = std::min(al, L - lo);
        long tot = (long)nct << c->logN;  // one thread per (ciphertext, coefficient)
        {
            ProfScope ps(c, "modup", 8.0 * c->N * ((double)nct * 2 * ds + (double)nct * nl));
            klaunch(k_modup, grid_for(c, tot), 256, 0, c->st)(dig.get(), (long)nd * nl * c->N, (long)j * nl * c->N,
                                                          tmp.get(), (long)L * c->N, nct, lo, ds, nl, em, c->d_mods,
                                                          c->d_cv + c->cv_off[L - 1][j], c->logN, x, sx);
        }
        LAUNCH_CHECK();
        // forward NTT of the limbs outside the digit: [0, lo) and [lo + ds, L + alpha)
        const int ranges[2][2] = {{0, lo}, {lo + ds, nl}};
        for (const auto &r : ranges) {
            int a = r[0], b = r[1];
            if (b <= a) continue;
            LimbMap sub;
            sub.nper = b - a;
            for (int t = a; t < b; t++) sub.prime[t - a] = em.prime[t];
            ntt(c, dig.get() + (long)j * nl * c->N + (long)a * c->N, nct * (b - a), sub, (long)nd * nl * c->N, false,
                "ntt_modup");
        }
    }
    return dig;
}

// key-switch inner product sum_j d~_j swk_j over Q_l u P (automorphism g applied to the digits
// when g > 1) into acc [nct][2][L + alpha][N] (NTT form); accumulate: added to acc
static void ks_inner_into(he_ctx *c, uint64_t *acc, const uint64_t *dig, int nct, int L, int g, const uint64_t *key,
                          bool accumulate) {
    int al = c->alpha, nd = (L + al - 1) / al, nl = L + al;
    {
        ProfScope ps(c, "ks_inner", 8.0 * c->N * ((double)nct * nd * nl + 2.0 * nd * nl + 2.0 * nct * nl *
                                                                            (accumulate ? 2 : 1)));
        KsMulti M{};
        launch_ks_inner(grid_for(c, (long)nl << c->logN), c->st, acc, dig, nct, nd, L, al, extmap(c, L), c->d_mods, key,
                        c->nm, c->nq, g, c->logN, accumulate ? 1 : 0, M);
    }
    LAUNCH_CHECK();
    c->cnt[0] += nct;  // ciphertext key switches (a batch of nct counts nct)
}

// ModDown of acc (its P limbs are transformed in place) into out (nct ciphertexts at level
// L-1, stride so); when add is given (it may be out itself) its two polynomials (ciphertext
// stride sadd) are added to the result
static void ks_moddown(he_ctx *c, uint64_t *acc, int nct, int L, uint64_t *out, long so, const uint64_t *add,
                       long sadd) {
    int al = c->alpha, nl = L + al;
    // P limbs to coefficient form, times N^{-1} [phat_k^{-1}]_{p_k} (the conversion's first factor)
    ntt(c, acc + (long)L * c->N, 2 * nct * al, pmap(c), (long)nl * c->N, true, "ntt_moddown", nullptr, 0, nullptr,
        c->d_ninv_down);
    DPtr conv = dalloc(c, (size_t)2 * nct * L * c->N);
    if (tune_pick(c, HE_TUNE_FUSE_CONV, L, nct, 0)) {
        // Conv_{P->Q} in the transform's column pass (kind 5), (x - conv) P^{-1} (+ add) in its
        // row pass; conv only carries the column pass's output to the row pass
        NttFuse F{};
        F.kind = 5;
        F.alpha = al;
        F.x = acc;
        F.out = out;
        F.so = so;
        F.add = add;
        F.sadd = sadd;
        F.cst = c->d_pinv;
        F.src = acc;
        F.sstride = (long)nl * c->N;
        F.slo = L;
        F.ns = al;
        for (int k = 0; k < al; k++) F.sidx[k] = c->nq + k;
        F.cvw = c->d_mdcv + 2 * al;
        F.wstride = c->nq;
        ntt(c, conv.get(), 2 * nct * L, qmap(L), (long)L * c->N, false, "ntt_moddown", nullptr, 0, &F);
        return;
    }
    {
        ProfScope ps_(c, "moddown", 8.0 * c->N * 2 * nct * (al + L));
        klaunch(k_moddown_conv, grid_for(c, (long)2 * nct << c->logN), 256, 0, c->st)(conv.get(), acc, 2 * nct, L, al, qmap(L),
                                                                                  c->d_pidx, c->d_mods, c->d_mdcv,
                                                                                  c->nq, c->logN);
    }
    LAUNCH_CHECK();
    // (x - conv) P^{-1} (+ add) fused into the transform of conv
    NttFuse F{};
    F.kind = 1;
    F.alpha = al;
    F.x = acc;
    F.out = out;
    F.so = so;
    F.add = add;
    F.sadd = sadd;
    F.cst = c->d_pinv;
    ntt(c, conv.get(), 2 * nct * L, qmap(L), (long)L * c->N, false, "ntt_moddown", nullptr, 0, &F);
}

// one key switch: inner product and ModDown into out (see ks_moddown for add)
static void ks_finish(he_ctx *c, const uint64_t *dig, int nct, int L, int g, const uint64_t *key, uint64_t *out,
                      long so, const uint64_t *add, long sadd) {
    int nl = L + c->alpha;
    DPtr acc = dalloc(c, (size_t)nct * 2 * nl * c->N);
    ks_inner_into(c, acc.get(), dig, nct, L, g, key, false);
    ks_moddown(c, acc.get(), nct, L, out, so, add, sadd);
}

static const uint64_t *get_key(he_ctx *c, int galois) {
    auto it = c->keys.find(galois);
    if (it == c->keys.end()) {
        char b[96];
        snprintf(b, sizeof b, "no evaluation key for galois element %d", galois);
        throw HeErr{HE_ENOKEY, b};
    }
    return it->second;
}

// d: [nct][3][L][N] (ct stride 3 L N) -> ciphertexts (d0 + k0, d1 + k1), scale given
static DCt relinearize(he_ctx *c, const uint64_t *d, int level, int nct, double scale) {
    int L = level + 1;
    DCt y = ct_new(c, level, nct, scale);
    DPtr dig = ks_modup(c, d + 2L * L * c->N, 3L * L * c->N, nct, L);
    // y = (d0, d1) + KS(d2): d0 and d1 are added by the ModDown epilogue
    ks_finish(c, dig.get(), nct, L, 0, get_key(c, 0), y.d, y.cs(c), d, 3L * L * c->N);
    return y;
}

// Relinearisation and rescale as one division by P q_l: K = KS(d2) over Q_l u P,
// Y = P (d0, d1) + K, out_i = (Y_i - Conv_{D->q_i}([Y]_D)) (P q_l)^{-1} with D = {q_l} u P
// (the dropped limbs l .. l + alpha of Y, contiguous).  d: [nct][3][l+1][N] NTT form.
static DCt relin_rescale(he_ctx *c, const uint64_t *d, int level, int nct, double scale) {
    int l = level, L = l + 1, al = c->alpha, nl = L + al, nd = al + 1;
    REQUIRE(l >= 1, HE_ELEVEL, "relinearise + rescale at level 0");
    DPtr dig = ks_modup(c, d + 2L * L * c->N, 3L * L * c->N, nct, L);
    DPtr acc = dalloc(c, (size_t)nct * 2 * nl * c->N);
    ks_inner_into(c, acc.get(), dig.get(), nct, L, 0, get_key(c, 0), false);
    dig.reset();
    // Y_l = K_l + P d_l (P d vanishes mod every p_k); polynomials 0 and 1 of every ciphertext
    Scal pm;
    {
        uint64_t q = c->mods[l], v = 1 % q;
        for (int k = 0; k < al; k++) v = h_mulmod(v, c->mods[c->nq + k] % q, q);
        pm.v[0] = v;
    }
    for (int p = 0; p < 2; p++) {
        {
            ProfScope ps_(c, "elementwise", 0);
            klaunch(k_axpy_scalar, grid_for(c, (long)nct << c->logN), 256, 0, c->st)(
                acc.get() + (long)p * nl * c->N + (long)l * c->N, 2L * nl * c->N, d + (long)p * L * c->N + (long)l * c->N,
                3L * L * c->N, pm, nct, 1, single(l), c->d_mods, c->logN);
        }
        LAUNCH_CHECK();
    }
    // the dropped limbs to coefficient form, converted to q_0 .. q_{l-1}
    LimbMap dm;
    dm.nper = nd;
    dm.prime[0] = l;
    for (int k = 0; k < al; k++) dm.prime[1 + k] = c->nq + k;
    ntt(c, acc.get() + (long)l * c->N, 2 * nct * nd, dm, (long)nl * c->N, true, "ntt_moddown", nullptr, 0, nullptr,
        c->d_ninv_rr + (size_t)l * 2 * c->nm);
    DPtr conv = dalloc(c, (size_t)2 * nct * l * c->N);
    DCt y = ct_new(c, l - 1, nct, scale / (double)c->mods[l]);
    const uint64_t *cst = c->d_rrpq + (size_t)l * c->nq * 4;
    NttFuse F{};
    F.kind = 3;
    F.alpha = nd;
    F.x = acc.get();
    F.add = d;
    F.sadd = 3L * L * c->N;
    F.out = y.d;
    F.so = y.cs(c);
    F.cst = cst;
    if (tune_pick(c, HE_TUNE_FUSE_CONV, L, nct, 0)) {
        // Conv_{D->Q} in the column pass (kind 6), the division in the row pass
        F.kind = 6;
        F.src = acc.get();
        F.sstride = (long)nl * c->N;
        F.slo = l;
        F.ns = nd;
        for (int j = 0; j < nd; j++) F.sidx[j] = j == 0 ? l : c->nq + (j - 1);
        F.cvw = c->d_rrcv + (size_t)l * c->rrcv_stride + 2 * nd;
        F.wstride = c->nq;
        ntt(c, conv.get(), 2 * nct * l, qmap(l), (long)l * c->N, false, "ntt_moddown", nullptr, 0, &F);
        c->cnt[3]++;
        return y;
    }
    {
        ProfScope ps_(c, "moddown", 8.0 * c->N * 2 * nct * (nd + l));
        klaunch(k_moddown_conv, grid_for(c, (long)2 * nct << c->logN), 256, 0, c->st)(
            conv.get(), acc.get(), 2 * nct, l, nd, qmap(l), c->d_rridx + (size_t)l * nd, c->d_mods,
            c->d_rrcv + (size_t)l * c->rrcv_stride, c->nq, c->logN);
    }
    LAUNCH_CHECK();
    ntt(c, conv.get(), 2 * nct * l, qmap(l), (long)l * c->N, false, "ntt_moddown", nullptr, 0, &F);
    c->cnt[3]++;
    return y;
}

// d[i] = a[i] (x) b[i / bdiv] for the a.nct ciphertexts of a (bdiv = a.nct: b's one ciphertext
// with every one of a), limbs 0..level of each
static void tensor_into(he_ctx *c, uint64_t *d, const DCt &a, const DCt &b, int level, bool accumulate, int bdiv = 1) {
    int L = level + 1;
    long tot = (long)a.nct * L << c->logN;
    ProfScope ps(c, "tensor", 8.0 * c->N * L * ((double)a.nct * (2 + 3) + 2.0 * (a.nct / bdiv)));
    klaunch(k_tensor, grid_for(c, tot), 256, 0, c->st)(d, 3L * L * c->N, a.d, a.cs(c), b.d, b.cs(c), b.ps(c), bdiv, a.nct, L,
                                                   qmap(L), c->d_mods, c->logN, accumulate ? 1 : 0);
    LAUNCH_CHECK();
}

// tensor, relinearise, rescale; operands at different levels: the higher one is dropped
static DCt hmult(he_ctx *c, const DCt &a, const DCt &b) {
    int level = std::min(a.level, b.level);
    REQUIRE(level >= 1, HE_ELEVEL, "hmult at level 0");
    REQUIRE(a.nct == b.nct || b.nct == 1 || a.nct == 1, HE_EINVAL, "hmult: batch sizes");
    int nct = std::max(a.nct, b.nct);
    DPtr d = dalloc(c, (size_t)nct * 3 * (level + 1) * c->N);
    if (a.nct == b.nct) {
        tensor_into(c, d.get(), a, b, level, false);
    } else {
        // one operand shared by every ciphertext of the other batch: one launch
        const DCt &many = a.nct > 1 ? a : b, &one = a.nct > 1 ? b : a;
        tensor_into(c, d.get(), many, one, level, false, many.nct);
    }
    DCt r = relin_rescale(c, d.get(), level, nct, a.scale * b.scale);
    c->cnt[2]++;
    return r;
}

// lam (G ciphertexts) times y (G groups of m ciphertexts): ciphertext i of y with lam[i / m]
static DCt hmult_grouped(he_ctx *c, const DCt &lam, const DCt &y, int m) {
    int level = std::min(lam.level, y.level);
    REQUIRE(level >= 1, HE_ELEVEL, "hmult at level 0");
    REQUIRE(y.nct == lam.nct * m, HE_EINVAL, "hmult_grouped: batch sizes");
    DPtr d = dalloc(c, (size_t)y.nct * 3 * (level + 1) * c->N);
    tensor_into(c, d.get(), y, lam, level, false, m);   // ciphertext i of y with lam[i / m], one launch
    DCt r = relin_rescale(c, d.get(), level, y.nct, lam.scale * y.scale);
    c->cnt[2]++;
    return r;
}

// Rot by galois elements: ModUp(c1) once, then for every g: X -> X^g on the digits and c0,
// inner product with swk(s(X^g) -> s), ModDown.
// y.c0 += x.c0(X^g) for every ciphertext of the batch
static void automorph_acc(he_ctx *c, DCt &y, const DCt &x, int g) {
    int L = x.level + 1;
    long tot = (long)x.nct * L << c->logN;
    {
        ProfScope ps_(c, "automorph", 0);
        klaunch(k_automorph_acc, grid_for(c, tot), 256, 0, c->st)(y.d, y.cs(c), x.d, x.cs(c), x.nct * L, L, qmap(L),
                                                              c->d_mods, g, c->logN);
    }
    LAUNCH_CHECK();
}

static std::vector<DCt> rotate_hoisted(he_ctx *c, const DCt &x, const std::vector<int> &gal) {
    int L = x.level + 1;
    std::vector<DCt> out;
    DPtr dig;
    bool need = false;
    for (int g : gal) need |= g != 1;
    if (need) dig = ks_modup(c, x.d + (long)L * c->N, x.cs(c), x.nct, L);
    std::vector<int> gs;
    for (int g : gal)
        if (g != 1) gs.push_back(g);
    if (gs.size() >= 2 && gs.size() <= 16 && tune_pick(c, HE_TUNE_ROT, L, x.nct, x.nct <= 4)) {
        // small batches: the key switches of all rotations in one inner-product launch and one
        // ModDown over all of them (each separately would fill a fraction of the GPU)
        int al = c->alpha, nd = (L + al - 1) / al, nl = L + al, ng = (int)gs.size();
        KsMulti M{};
        M.n = ng;
        M.acc_stride = (long)x.nct * 2 * nl * c->N;
        for (int r = 0; r < ng; r++) {
            M.key[r] = get_key(c, gs[r]);
            M.g[r] = gs[r];
        }
        DPtr acc = dalloc(c, (size_t)ng * M.acc_stride);
        {
            ProfScope ps(c, "ks_inner", 8.0 * c->N * ng * ((double)x.nct * nd * nl + 2.0 * nd * nl + 2.0 * x.nct * nl));
            dim3 grid(grid_for(c, (long)nl << c->logN).x, ng);
            launch_ks_inner(grid, c->st, acc.get(), dig.get(), x.nct, nd, L, al, extmap(c, L), c->d_mods, nullptr, c->nm,
                            c->nq, 0, c->logN, 0, M);
        }
        LAUNCH_CHECK();
        c->cnt[0] += (long)ng * x.nct;
        long cs = x.cs(c);
        DPtr ys = dalloc(c, (size_t)ng * x.nct * cs);
        ks_moddown(c, acc.get(), ng * x.nct, L, ys.get(), cs, nullptr, 0);
        size_t r = 0;
        for (int g : gal) {
            if (g == 1) {
                out.push_back(ct_copy(c, x));
                continue;
            }
            DCt y;
            y.buf = ys;
            y.d = ys.get() + (long)r++ * x.nct * cs;
            y.level = x.level;
            y.scale = x.scale;
            y.nct = x.nct;
            automorph_acc(c, y, x, g);
            out.push_back(y);
            c->cnt[1]++;
        }
        return out;
    }
    for (int g : gal) {
        if (g == 1) {
            out.push_back(ct_copy(c, x));
            continue;
        }
        const uint64_t *key = get_key(c, g);
        DCt y = ct_new(c, x.level, x.nct, x.scale);
        // key switch of c1(X^g) written into y, then c0(X^g) added to its first polynomial
        ks_finish(c, dig.get(), x.nct, L, g, key, y.d, y.cs(c), nullptr, 0);
        automorph_acc(c, y, x, g);
        out.push_back(y);
        c->cnt[1]++;
    }
    return out;
}

static DCt rotate(he_ctx *c, const DCt &x, int g) { return rotate_hoisted(c, x, std::vector<int>{g})[0]; }

static int galois_for_rot(he_ctx *c, long r) {
    long n0 = c->n0, m = 2L * c->N;
    r %= n0;
    if (r < 0) r += n0;
    long g = 1;
    for (long i = 0; i < r; i++) g = (g * 5) % m;
    return (int)g;
}

static DCt mod_raise(he_ctx *c, const DCt &a, int top) {
    REQUIRE(a.level == 0, HE_EINVAL, "mod_raise needs level 0");
    int npoly = 2 * a.nct, L = top + 1;
    DPtr x0 = dalloc(c, (size_t)npoly * c->N);
    ntt(c, x0.get(), npoly, single(0), c->N, true, "ntt_modraise", a.d, c->N);
    DCt y = ct_new(c, top, a.nct, a.scale);
    long tot = (long)npoly * L << c->logN;
    {
        ProfScope ps_(c, "modraise", 0);
        klaunch(k_modraise, grid_for(c, tot), 256, 0, c->st)(y.d, x0.get(), npoly, L, qmap(L), c->d_mods, c->mods[0], c->logN);
    }
    LAUNCH_CHECK();
    ntt(c, y.d, npoly * L, qmap(L), (long)L * c->N, false, "ntt_modraise");
    return y;
}

// ------------------------------------------------------------------------- encoding
// slots z (N0 complex, host) -> plaintext round(scale t) in NTT form, limbs 0..level
static DPtr encode(he_ctx *c, const std::vector<double2> &z, double scale, int level) {
    int n0 = c->n0, L = level + 1;
    DPtr w = dalloc(c, (size_t)2 * n0);
    double2 *wd = (double2 *)w.get();
    CK(cudaMemcpyAsync(wd, z.data(), sizeof(double2) * n0, cudaMemcpyHostToDevice, c->st));
    dim3 g = grid_for(c, n0 / 2);
    {
        ProfScope ps_(c, "encode", 0);
        for (int len = n0; len >= 2; len >>= 1)
            klaunch(k_sfft_inv_stage, g, 256, 0, c->st)(wd, n0, len, c->d_zeta, c->d_rg, 2 * c->N);
        klaunch(k_bitrev_c, grid_for(c, n0), 256, 0, c->st)(wd, n0, c->logN - 1);
        klaunch(k_scale_c, grid_for(c, n0), 256, 0, c->st)(wd, n0, (double)n0);
    }
    LAUNCH_CHECK();
    DPtr pt = dalloc(c, (size_t)L * c->N);
    {
        ProfScope ps_(c, "encode", 0);
        klaunch(k_round_to_limbs, grid_for(c, (long)L << c->logN), 256, 0, c->st)(pt.get(), 0, wd, scale, L, L, qmap(L),
                                                                             c->d_mods, c->logN);
    }
    LAUNCH_CHECK();
    ntt(c, pt.get(), L, qmap(L), (long)L * c->N, false);
    return pt;
}

// device small integers (signed) -> NTT-form residues for the limbs of map
static void small_to_ntt(he_ctx *c, uint64_t *out, const int64_t *v, const LimbMap &m) {
    {
        ProfScope ps_(c, "encode", 0);
        klaunch(k_small_to_limbs, grid_for(c, (long)m.nper << c->logN), 256, 0, c->st)(out, 0, v, m.nper, m.nper, m, c->d_mods,
                                                                                   c->logN);
    }
    LAUNCH_CHECK();
    ntt(c, out, m.nper, m, (long)m.nper * c->N, false);
}

enum { DOM_SK = 1, DOM_SK_SIGN = 2, DOM_PK_A = 3, DOM_PK_E = 4, DOM_ENC_V = 5, DOM_ENC_E0 = 6, DOM_ENC_E1 = 7 };
static uint64_t dom_key(int key_id, int digit, int which) {
    return 0x100000ULL + ((uint64_t)key_id * 256ULL + (uint64_t)digit) * 2ULL + (uint64_t)which;
}

static void sample_small(he_ctx *c, int64_t *out, uint64_t seed, uint64_t dom, uint64_t ctr0, int kind) {
    {
        ProfScope ps_(c, "keygen", 0);
        klaunch(k_sample_small, grid_for(c, c->N), 256, 0, c->st)(out, c->N, seed, dom, ctr0, c->d_cdt, c->cdt_len, kind);
    }
    LAUNCH_CHECK();
}

static void encrypt_into(he_ctx *c, const std::vector<double2> &z, int level, double scale, uint64_t seed, int ct_index,
                         uint64_t *out) {
    REQUIRE(c->have_keys, HE_ENOKEY, "encrypt before keygen");
    int L = level + 1;
    DPtr pt = encode(c, z, scale, level);
    DPtr sm = dalloc(c, 3 * (size_t)c->N);
    int64_t *v = (int64_t *)sm.get(), *e0 = v + c->N, *e1 = e0 + c->N;
    uint64_t ctr = (uint64_t)ct_index * c->N;
    sample_small(c, v, seed, DOM_ENC_V, ctr, 1);
    sample_small(c, e0, seed, DOM_ENC_E0, ctr, 0);
    sample_small(c, e1, seed, DOM_ENC_E1, ctr, 0);
    DPtr lv = dalloc(c, 3 * (size_t)L * c->N);
    uint64_t *vn = lv.get(), *e0n = vn + (long)L * c->N, *e1n = e0n + (long)L * c->N;
    LimbMap m = qmap(L);
    small_to_ntt(c, vn, v, m);
    small_to_ntt(c, e0n, e0, m);
    small_to_ntt(c, e1n, e1, m);
    long tot = (long)L << c->logN;
    uint64_t *c0 = out, *c1 = out + (long)L * c->N;
    const uint64_t *pkb = c->d_pk, *pka = c->d_pk + (long)c->nq * c->N;
    {
        ProfScope ps_(c, "elementwise", 0);
        klaunch(k_mul, grid_for(c, tot), 256, 0, c->st)(c0, 0, vn, 0, pkb, 0, L, L, m, c->d_mods, c->logN, 0);
    }
    {
        ProfScope ps_(c, "elementwise", 0);
        klaunch(k_mul, grid_for(c, tot), 256, 0, c->st)(c1, 0, vn, 0, pka, 0, L, L, m, c->d_mods, c->logN, 0);
    }
    {
        ProfScope ps_(c, "elementwise", 0);
        klaunch(k_add, grid_for(c, tot), 256, 0, c->st)(c0, 0, c0, 0, e0n, 0, L, L, m, c->d_mods, c->logN, 0);
    }
    {
        ProfScope ps_(c, "elementwise", 0);
        klaunch(k_add, grid_for(c, tot), 256, 0, c->st)(c0, 0, c0, 0, pt.get(), 0, L, L, m, c->d_mods, c->logN, 0);
    }
    {
        ProfScope ps_(c, "elementwise", 0);
        klaunch(k_add, grid_for(c, tot), 256, 0, c->st)(c1, 0, c1, 0, e1n, 0, L, L, m, c->d_mods, c->logN, 0);
    }
    LAUNCH_CHECK();
}

static std::vector<double2> decrypt_slots(he_ctx *c, const DCt &x, int i) {
    REQUIRE(c->have_keys, HE_ENOKEY, "decrypt before keygen");
    int L = x.level + 1;
    const uint64_t *c0 = x.d + (long)i * x.cs(c), *c1 = c0 + (long)L * c->N;
    DPtr m = dalloc(c, (size_t)L * c->N);
    long tot = (long)L << c->logN;
    {
        ProfScope ps_(c, "elementwise", 0);
        klaunch(k_mul, grid_for(c, tot), 256, 0, c->st)(m.get(), 0, c1, 0, c->d_s, 0, L, L, qmap(L), c->d_mods, c->logN, 0);
    }
    {
        ProfScope ps_(c, "elementwise", 0);
        klaunch(k_add, grid_for(c, tot), 256, 0, c->st)(m.get(), 0, m.get(), 0, c0, 0, L, L, qmap(L), c->d_mods, c->logN, 0);
    }
    LAUNCH_CHECK();
    ntt(c, m.get(), L, qmap(L), (long)L * c->N, true);
    DPtr w = dalloc(c, (size_t)2 * c->n0);
    double2 *wd = (double2 *)w.get();
    {
        ProfScope ps_(c, "decode", 0);
        klaunch(k_crt_to_double, grid_for(c, c->N), 128, 0, c->st)(wd, m.get(), L, qmap(L), c->d_mods, c->d_radix, c->d_radinv,
                                                              c->d_qd, x.scale, c->logN);
    }
    {
        ProfScope ps_(c, "decode", 0);
        klaunch(k_bitrev_c, grid_for(c, c->n0), 256, 0, c->st)(wd, c->n0, c->logN - 1);
        for (int len = 2; len <= c->n0; len <<= 1)
            klaunch(k_sfft_fwd_stage, grid_for(c, c->n0 / 2), 256, 0, c->st)(wd, c->n0, len, c->d_zeta, c->d_rg, 2 * c->N);
    }
    LAUNCH_CHECK();
    std::vector<double2> z(c->n0);
    CK(cudaMemcpyAsync(z.data(), wd, sizeof(double2) * c->n0, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return z;
}

// ------------------------------------------------------------------------- key generation
static void keygen(he_ctx *c, uint64_t seed) {
    c->seed = seed;
    int N = c->N, nm = c->nm;
    DPtr sint = dalloc(c, N);
    {
        ProfScope ps_(c, "keygen", 0);
        klaunch(k_sample_hwt, (N + 255) / 256, 256, 256 * 8, c->st)((int64_t *)sint.get(), N, c->h, seed, DOM_SK, DOM_SK_SIGN);
    }
    LAUNCH_CHECK();
    if (!c->d_s) CK(cudaMalloc(&c->d_s, (size_t)nm * N * 8));
    small_to_ntt(c, c->d_s, (int64_t *)sint.get(), allmap(c));
    // public key over Q
    if (!c->d_pk) CK(cudaMalloc(&c->d_pk, (size_t)2 * c->nq * N * 8));
    uint64_t *pkb = c->d_pk, *pka = c->d_pk + (long)c->nq * N;
    DPtr e = dalloc(c, N), el = dalloc(c, (size_t)nm * N);
    sample_small(c, (int64_t *)e.get(), seed, DOM_PK_E, 0, 0);
    LimbMap qm = qmap(c->nq);
    small_to_ntt(c, el.get(), (int64_t *)e.get(), qm);
    {
        ProfScope ps_(c, "keygen", 0);
        klaunch(k_sample_uniform, grid_for(c, (long)c->nq << c->logN), 256, 0, c->st)(pka, 0, c->nq, c->nq, qm, c->d_mods, seed,
                                                                                  DOM_PK_A, c->logN);
    }
    LAUNCH_CHECK();
    ntt(c, pka, c->nq, qm, (long)c->nq * N, false);
    Scal z0;
    memset(&z0, 0, sizeof z0);
    {
        ProfScope ps_(c, "keygen", 0);
        klaunch(k_key_combine, grid_for(c, (long)c->nq << c->logN), 256, 0, c->st)(pkb, pka, el.get(), c->d_s, nullptr, z0, c->nq,
                                                                               0, 0, qm, c->d_mods, c->logN);
    }
    LAUNCH_CHECK();
    c->have_keys = true;
}

static void make_key(he_ctx *c, int galois) {
    if (c->keys.count(galois)) return;
    int N = c->N, nm = c->nm, nd = c->ndig_top;
    uint64_t *key = nullptr;
    CK(cudaMalloc(&key, (size_t)nd * 2 * nm * N * 8));
    LimbMap am = allmap(c);
    DPtr sp = dalloc(c, (size_t)nm * N), e = dalloc(c, N), el = dalloc(c, (size_t)nm * N);
    long tot = (long)nm << c->logN;
    if (galois == 0)
        {
            ProfScope ps_(c, "elementwise", 0);
            klaunch(k_mul, grid_for(c, tot), 256, 0, c->st)(sp.get(), 0, c->d_s, 0, c->d_s, 0, nm, nm, am, c->d_mods, c->logN, 0);
        }
    else
        {
            ProfScope ps_(c, "automorph", 0);
            klaunch(k_automorph, grid_for(c, tot), 256, 0, c->st)(sp.get(), 0, c->d_s, 0, nm, nm, galois, c->logN);
        }
    LAUNCH_CHECK();
    Scal pm;
    for (int t = 0; t < nm; t++) {
        uint64_t q = c->mods[t], v = 1 % q;
        for (int k = 0; k < c->np; k++) v = h_mulmod(v, c->mods[c->nq + k] % q, q);
        pm.v[t] = v;
    }
    for (int j = 0; j < nd; j++) {
        uint64_t *b = key + (size_t)(2 * j) * nm * N, *a = key + (size_t)(2 * j + 1) * nm * N;
        sample_small(c, (int64_t *)e.get(), c->seed, dom_key(galois, j, 1), 0, 0);
        small_to_ntt(c, el.get(), (int64_t *)e.get(), am);
        {
            ProfScope ps_(c, "keygen", 0);
            klaunch(k_sample_uniform, grid_for(c, tot), 256, 0, c->st)(a, 0, nm, nm, am, c->d_mods, c->seed, dom_key(galois, j, 0),
                                                                   c->logN);
        }
        LAUNCH_CHECK();
        ntt(c, a, nm, am, (long)nm * N, false);
        int dlo = j * c->alpha, dhi = std::min((j + 1) * c->alpha, c->nq);
        {
            ProfScope ps_(c, "keygen", 0);
            klaunch(k_key_combine, grid_for(c, tot), 256, 0, c->st)(b, a, el.get(), c->d_s, sp.get(), pm, nm, dlo, dhi, am,
                                                                c->d_mods, c->logN);
        }
        LAUNCH_CHECK();
    }
    // stored in Montgomery form (k 2^64 mod q): the inner product sums raw 128-bit products
    // and reduces once
    Scal rm;
    for (int t = 0; t < nm; t++) rm.v[t] = h_mont(1, c->mods[t]);
    {
        ProfScope ps_(c, "elementwise", 0);
        klaunch(k_mul_scalar, grid_for(c, (long)2 * nd * nm << c->logN), 256, 0, c->st)(key, (long)nm * N, key, (long)nm * N, rm, 2 * nd * nm, nm, am,
                                                                                  c->d_mods, c->logN);
    }
    LAUNCH_CHECK();
    c->keys[galois] = key;
}

// ------------------------------------------------------------------------- polynomial evaluation
// Chebyshev evaluation with exact scale targets (same recursion and constants as the
// reference definition): see eval() below.
struct PolyEval {
    he_ctx *c;
    std::map<int, DCt> T;
    int lin;

    DCt adjust(const DCt &x, int lt, double st) {
        REQUIRE(x.level >= lt + 1, HE_ELEVEL, "adjust: level");
        int L = lt + 2;
        double q = (double)c->mods[lt + 1];
        // drop to level lt + 1 and multiply by the integer in one pass
        DCt y = ct_new(c, lt + 1, x.nct, st * q);
        Scal s = scal_of(c, h_round((st * q) / x.scale), L);
        {
            ProfScope ps_(c, "elementwise", 0);
            klaunch(k_mul_scalar, grid_for(c, (long)2 * x.nct * L << c->logN), 256, 0, c->st)(
                y.d, y.ps(c), x.d, x.ps(c), s, 2 * x.nct * L, L, qmap(L), c->d_mods, c->logN);
        }
        LAUNCH_CHECK();
        return rescale(c, y);
    }

    const DCt &getT(int k) {
        auto it = T.find(k);
        if (it != T.end()) return it->second;
        REQUIRE(k >= 1, HE_EINVAL, "getT");
        // inside a branch every basis element must exist already (precompute): one made here could
        // be read by another branch before this one is joined
        REQUIRE(c->branch_depth == 0, HE_EINVAL, "polynomial evaluation: basis element not precomputed");
        if ((k & (k - 1)) == 0) {
            const DCt &h = getT(k / 2);
            DCt x = hmult(c, h, h);
            ct_mul_int(c, x, 2);
            ct_add_const(c, x, h_round(-x.scale));
            T[k] = x;
        } else {
            int a = 1;
            while (a * 2 < k) a *= 2;
            int b = k - a;
            getT(a);
            getT(b);
            getT(a - b);
            DCt p = hmult(c, T[a], T[b]);
            ct_mul_int(c, p, 2);
            DCt s = adjust(T[a - b], p.level, p.scale);
            ct_add_inplace(c, p, s, true);
            T[k] = p;
        }
        return T[k];
    }

    static int trim(const std::vector<double> &cf, int d) {
        while (d > 0 && cf[d] == 0.0) d--;
        return d;
    }

    // the basis elements T_k that eval(cf_in, d, lt, .) reads, walking its recursion on the host
    void collect(const std::vector<double> &cf_in, int d, int lt, std::set<int> &need) const {
        d = trim(cf_in, d);
        if (d < 1) return;
        int avail = lin - lt, j = ilog2c(d + 1);
        if (d < 8 && avail >= ilog2c(d) + 1) {
            for (int k = 1; k <= d; k++)
                if (cf_in[k] != 0.0) need.insert(k);
            return;
        }
        int a = 1 << (j - 1);
        std::vector<double> q(d - a + 1, 0.0), r(a, 0.0);
        split(cf_in, d, a, q, r);
        need.insert(a);
        int dq = trim(q, d - a);
        if (dq != 0) collect(q, dq, lt + 1, need);
        int dr = trim(r, a - 1);
        if (dr >= 1) collect(r, dr, lt, need);
    }

    // Chebyshev division p = r + T_a q (T_i = 2 T_a T_(i-a) - T_(2a-i)): q, r from the coefficients
    static void split(const std::vector<double> &cf_in, int d, int a, std::vector<double> &q, std::vector<double> &r) {
        q[0] = cf_in[a];
        for (int i = 1; i <= d - a; i++) q[i] = 2.0 * cf_in[a + i];
        for (int i = 0; i < a; i++) r[i] = cf_in[i];
        for (int i = a + 1; i <= d; i++) r[2 * a - i] = r[2 * a - i] - cf_in[i];
    }

    static void deps(int k, int *dk, int &nd) {
        nd = 0;
        if ((k & (k - 1)) == 0) {
            dk[nd++] = k / 2;
            return;
        }
        int a = 1;
        while (a * 2 < k) a *= 2;
        dk[nd++] = a;
        dk[nd++] = k - a;
        dk[nd++] = a - (k - a);
    }

    // makes every T_k of need and their dependencies, layer by layer (a layer's elements depend
    // only on earlier layers); the elements of one layer are computed concurrently, one on the
    // main stream and the others on side streams
    void precompute(std::set<int> need) {
        std::vector<int> todo(need.begin(), need.end());
        while (!todo.empty()) {   // closure under deps
            int k = todo.back();
            todo.pop_back();
            int dk[3], nd;
            if (k <= 1) continue;
            deps(k, dk, nd);
            for (int i = 0; i < nd; i++)
                if (dk[i] >= 1 && !need.count(dk[i])) {
                    need.insert(dk[i]);
                    todo.push_back(dk[i]);
                }
        }
        std::map<int, int> layer;
        layer[1] = 0;
        int maxl = 0;
        for (int k : need) {   // ascending: dependencies are smaller
            if (k <= 1) continue;
            int dk[3], nd, l = 0;
            deps(k, dk, nd);
            for (int i = 0; i < nd; i++) l = std::max(l, layer.count(dk[i]) ? layer[dk[i]] : 0);
            layer[k] = l + 1;
            maxl = std::max(maxl, l + 1);
        }
        for (int l = 1; l <= maxl; l++) {
            std::vector<int> ks;
            for (int k : need)
                if (k > 1 && layer[k] == l && !T.count(k)) ks.push_back(k);
            std::vector<std::unique_ptr<Branch>> br;
            for (size_t i = 1; i < ks.size(); i++) br.emplace_back(new Branch(c));   // all fork here
            for (size_t i = 0; i < ks.size(); i++) {
                if (i > 0) br[i - 1]->enter();
                T[ks[i]] = makeT(ks[i]);
                if (i > 0) br[i - 1]->leave();
            }
            for (auto &b : br) b->join();
        }
    }

    // T_k from its dependencies (all present)
    DCt makeT(int k) {
        if ((k & (k - 1)) == 0) {
            const DCt &h = T.at(k / 2);
            DCt x = hmult(c, h, h);
            ct_mul_int(c, x, 2);
            ct_add_const(c, x, h_round(-x.scale));
            return x;
        }
        int a = 1;
        while (a * 2 < k) a *= 2;
        int b = k - a;
        DCt p = hmult(c, T.at(a), T.at(b));
        ct_mul_int(c, p, 2);
        DCt s = adjust(T.at(a - b), p.level, p.scale);
        ct_add_inplace(c, p, s, true);
        return p;
    }

    // sum_k round(cf_k st q / scale_k) T_k + round(cf_0 st q) at level lt + 1, then rescale:
    // one pass over the T_k (drop, integer products, sum and constant fused)
    DCt lincomb(const std::vector<double> &cf, int d, int lt, double st) {
        double q = (double)c->mods[lt + 1];
        int L = lt + 2;
        for (int k = 1; k <= d; k++)
            if (cf[k] != 0.0) getT(k);
        LcArgs A;
        memset(&A, 0, sizeof A);
        int nct = T[1].nct;
        for (int k = 1; k <= d; k++) {
            if (cf[k] == 0.0) continue;
            const DCt &tk = T[k];
            REQUIRE(tk.level >= lt + 1, HE_ELEVEL, "lincomb: level");
            REQUIRE(A.nt < HE_LC_MAXT, HE_EINVAL, "lincomb: too many terms");
            i128 kk = h_round(((cf[k] * st) * q) / tk.scale);
            for (int l = 0; l < L; l++) A.w[A.nt][l] = h_mont(h_red128(kk, c->mods[l]), c->mods[l]);
            A.x[A.nt] = tk.d;
            A.cs[A.nt] = tk.cs(c);
            A.ps[A.nt] = tk.ps(c);
            A.nt++;
        }
        REQUIRE(A.nt >= 1, HE_EINVAL, "lincomb: constant polynomial");
        i128 k0 = h_round((cf[0] * st) * q);
        for (int l = 0; l < L; l++) A.w[A.nt][l] = h_red128(k0, c->mods[l]);
        DCt out = ct_new(c, lt + 1, nct, st * q);
        {
            ProfScope ps_(c, "elementwise", 0);
            klaunch(k_lincomb, grid_for(c, (long)nct * 2 * L << c->logN), 256, 0, c->st)(out.d, A, nct, L, qmap(L),
                                                                                     c->d_mods, c->logN);
        }
        LAUNCH_CHECK();
        return rescale(c, out);
    }

    DCt eval(const std::vector<double> &cf_in, int d, int lt, double st) {
        d = trim(cf_in, d);
        REQUIRE(d >= 1, HE_EINVAL, "eval: degree 0");
        int avail = lin - lt;
        int j = ilog2c(d + 1);
        REQUIRE(avail >= j, HE_ELEVEL, "eval: not enough levels");
        if (d < 8 && avail >= ilog2c(d) + 1) return lincomb(cf_in, d, lt, st);
        int a = 1 << (j - 1);
        std::vector<double> q(d - a + 1, 0.0), r(a, 0.0);
        split(cf_in, d, a, q, r);
        getT(a);
        int dq = trim(q, d - a), dr = trim(r, a - 1);
        DCt out;
        // T_a q and r are independent: with both present, T_a q runs on a side stream beside r
        std::unique_ptr<Branch> bq(dq != 0 && dr >= 1 ? new Branch(c) : nullptr);
        if (bq) bq->enter();
        if (dq == 0) {
            std::vector<double> tmp(a + 1, 0.0);
            tmp[a] = q[0];
            out = lincomb(tmp, a, lt, st);
        } else {
            double sq = (st * (double)c->mods[lt + 1]) / T[a].scale;
            DCt Q = eval(q, dq, lt + 1, sq);
            out = hmult(c, T[a], Q);   // T_a's limbs above Q's level are not read
        }
        if (bq) bq->leave();
        if (dr >= 1) {
            DCt R = eval(r, dr, lt, st);
            if (bq) bq->join();
            ct_add_inplace(c, out, R);
        } else {
            ct_add_const(c, out, h_round(r[0] * out.scale));
        }
        return out;
    }
};

static DCt poly_eval(he_ctx *c, const DCt &u, const std::vector<double> &cf, int level_out, double scale_out) {
    PolyEval pe;
    pe.c = c;
    pe.T[1] = u;
    pe.lin = u.level;
    std::set<int> need;
    pe.collect(cf, (int)cf.size() - 1, level_out, need);
    pe.precompute(need);
    return pe.eval(cf, (int)cf.size() - 1, level_out, scale_out);
}

// ------------------------------------------------------------------------- linear transforms
// SlotToCoeff = butterfly stages of the special FFT (len = 2, 4, ..., N0) without the bit
// reversal; CoeffToSlot = their inverses in reverse order.  Stages are grouped into nlev
// levels of consecutive stages; each level is sum_d diag_d (.) Rot(x, d), evaluated by
// baby-step/giant-step with d = e hmin, e = a g + b.
struct LtDesc {
    int nstage;
    int h[32];
    int inverse;
};

static std::vector<LtDesc> lt_levels(he_ctx *c, int nlev, int inverse) {
    int s = c->logN - 1;
    std::vector<int> sizes(nlev);
    int base = s / nlev, rem = s % nlev;
    for (int g = 0; g < nlev; g++) sizes[g] = base + (g < rem ? 1 : 0);
    std::vector<LtDesc> fwd(nlev);
    int h = 1;
    for (int g = 0; g < nlev; g++) {
        fwd[g].nstage = sizes[g];
        fwd[g].inverse = 0;
        for (int k = 0; k < sizes[g]; k++) {
            fwd[g].h[k] = h;
            h <<= 1;
        }
    }
    if (!inverse) return fwd;
    std::vector<LtDesc> inv(nlev);
    for (int g = 0; g < nlev; g++) {
        const LtDesc &f = fwd[nlev - 1 - g];
        inv[g].nstage = f.nstage;
        inv[g].inverse = 1;
        for (int k = 0; k < f.nstage; k++) inv[g].h[k] = f.h[f.nstage - 1 - k];
    }
    return inv;
}

static double2 cmulh(double2 a, double2 b) {
    double2 r;
    double re = a.x * b.x - a.y * b.y;
    double im = a.x * b.y + a.y * b.x;
    r.x = re;
    r.y = im;
    return r;
}

static double2 lt_twiddle(he_ctx *c, int h, int j) {
    int lenq = 8 * h, m = 2 * c->N;
    return c->zeta[(c->rg[j] % lenq) * (m / lenq)];
}

static void lt_sources(he_ctx *c, int h, int inverse, int i, int *src, double2 *f) {
    int n0 = c->n0, pos = i % (2 * h);
    if (pos < h) {
        double2 t = lt_twiddle(c, h, pos);
        src[0] = i;
        src[1] = (i + h) % n0;
        if (!inverse) {
            f[0] = make_double2(1.0, 0.0);
            f[1] = t;
        } else {
            f[0] = make_double2(0.5, 0.0);
            f[1] = make_double2(0.5, 0.0);
        }
    } else {
        int j = pos - h;
        double2 t = lt_twiddle(c, h, j);
        src[0] = (i - h + n0) % n0;
        src[1] = i;
        if (!inverse) {
            f[0] = make_double2(1.0, 0.0);
            f[1] = make_double2(-t.x, -t.y);
        } else {
            f[0] = make_double2(t.x * 0.5, -(t.y * 0.5));
            f[1] = make_double2(-(t.x * 0.5), t.y * 0.5);
        }
    }
}

// plaintext [L][N] -> Montgomery form (x 2^64 mod q_l)
static void to_mont(he_ctx *c, uint64_t *pt, int L) {
    Scal rm;
    for (int l = 0; l < L; l++) rm.v[l] = h_mont(1, c->mods[l]);
    {
        ProfScope ps_(c, "elementwise", 0);
        klaunch(k_mul_scalar, grid_for(c, (long)L << c->logN), 256, 0, c->st)(pt, 0, pt, 0, rm, L, L, qmap(L), c->d_mods,
                                                                          c->logN);
    }
    LAUNCH_CHECK();
}

static int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
static int bsgs_g(int r) { return 1 << ((r + 2) / 2); }

static const LtLevel &lt_prepare(he_ctx *c, const LtDesc &lv, double gain, double pt_scale, int level) {
    char keyb[160];
    snprintf(keyb, sizeof keyb, "%d:%d:%d:%a:%a:%d", lv.inverse, lv.nstage, lv.h[0], gain, pt_scale, level);
    auto it = c->lt_cache.find(keyb);
    if (it != c->lt_cache.end()) return it->second;
    int n0 = c->n0, r = lv.nstage;
    int hmin = lv.h[0];
    for (int k = 1; k < r; k++) hmin = std::min(hmin, lv.h[k]);
    int E = (1 << r) - 1;
    std::vector<double2> diag((size_t)(2 * E + 1) * n0, make_double2(0.0, 0.0));
    std::vector<char> nz(2 * E + 1, 0);
    double2 gn = make_double2(gain, 0.0);
    for (int i = 0; i < n0; i++) {
        for (int path = 0; path < (1 << r); path++) {
            double2 fac[32];
            int idx = i;
            for (int k = r - 1; k >= 0; k--) {
                int src[2];
                double2 f[2];
                lt_sources(c, lv.h[k], lv.inverse, idx, src, f);
                int pick = (path >> k) & 1;
                fac[k] = f[pick];
                idx = src[pick];
            }
            double2 p = make_double2(1.0, 0.0);
            for (int k = 0; k < r; k++) p = cmulh(p, fac[k]);
            p = cmulh(p, gn);
            int off = ((idx - i) % n0 + n0) % n0;
            int e = off / hmin;
            if (e > E) e -= n0 / hmin;
            diag[(size_t)(e + E) * n0 + i] = p;
        }
    }
    for (int e = 0; e <= 2 * E; e++)
        for (int i = 0; i < n0 && !nz[e]; i++)
            if (diag[(size_t)e * n0 + i].x != 0.0 || diag[(size_t)e * n0 + i].y != 0.0) nz[e] = 1;
    LtLevel L;
    L.hmin = hmin;
    L.E = E;
    L.g = bsgs_g(r);
    std::vector<char> needb(L.g, 0);
    for (int e = -E; e <= E; e++)
        if (nz[e + E]) needb[e - floordiv(e, L.g) * L.g] = 1;
    for (int b = 0; b < L.g; b++)
        if (needb[b]) L.baby.push_back(b);
    std::vector<double2> rd(n0);
    for (int a = floordiv(-E, L.g); a <= floordiv(E, L.g); a++) {
        for (int b = 0; b < L.g; b++) {
            int e = a * L.g + b;
            if (e < -E || e > E || !nz[e + E]) continue;
            long sh = (long)a * L.g * hmin;
            const double2 *dv = diag.data() + (size_t)(e + E) * n0;
            for (int i = 0; i < n0; i++) rd[i] = dv[(((i - sh) % n0) + n0) % n0];
            LtPlain p;
            p.a = a;
            p.b = b;
            p.pt = encode(c, rd, pt_scale, level);
            to_mont(c, p.pt.get(), level + 1);   // read only by the fused inner sums
            L.pts.push_back(p);
        }
    }
    cache_entry_made(c);
    return c->lt_cache.emplace(keyb, std::move(L)).first->second;
}

static DCt lt_eval_level(he_ctx *c, const DCt &x, const LtDesc &lv, double gain, double pt_scale) {
    const LtLevel &Lv = lt_prepare(c, lv, gain, pt_scale, x.level);
    int L = x.level + 1;
    // baby steps Rot(x, b hmin), hoisted (one ModUp); b = 0 is x itself
    std::vector<int> gal;
    for (int b : Lv.baby)
        if (b != 0) gal.push_back(galois_for_rot(c, (long)b * Lv.hmin));
    std::vector<DCt> rots = rotate_hoisted(c, x, gal);
    LtArgs A;
    memset(&A, 0, sizeof A);
    std::map<int, int> bidx;
    size_t ri = 0;
    for (int b : Lv.baby) {
        REQUIRE(A.nb < HE_LT_MAXB, HE_EINVAL, "lintrans: too many baby steps");
        bidx[b] = A.nb;
        A.baby[A.nb++] = b == 0 ? x.d : rots[ri++].d;
    }
    // giant steps a (plaintexts are sorted by a): out_a = sum_b pt_{a,b} (.) baby_b in one pass;
    // small batches keep all the sums in one buffer (their c1 parts are then one ModUp batch)
    int na_max = 0;
    for (size_t pi = 0; pi < Lv.pts.size(); pi++)
        if (pi == 0 || Lv.pts[pi].a != Lv.pts[pi - 1].a) na_max++;
    const bool small = na_max >= 3 && na_max <= 17 && tune_pick(c, HE_TUNE_LT_SMALL, L, x.nct, x.nct <= 4);
    DPtr innerbuf = small ? dalloc(c, (size_t)na_max * x.nct * x.cs(c)) : DPtr();
    std::vector<int> gi;
    std::vector<DCt> inner;
    memset(A.ptix, -1, sizeof A.ptix);
    REQUIRE(Lv.pts.size() <= HE_LT_MAXPT, HE_EINVAL, "lintrans: too many diagonals");
    for (size_t pi = 0; pi < Lv.pts.size(); pi++) {
        int a = Lv.pts[pi].a;
        if (gi.empty() || gi.back() != a) {
            REQUIRE(gi.size() < HE_LT_MAXA, HE_EINVAL, "lintrans: too many giant steps");
            gi.push_back(a);
            if (small) {
                DCt v;
                v.buf = innerbuf;
                v.d = innerbuf.get() + (long)A.na * x.nct * x.cs(c);
                v.level = x.level;
                v.scale = x.scale * pt_scale;
                v.nct = x.nct;
                inner.push_back(v);
            } else {
                inner.push_back(ct_new(c, x.level, x.nct, x.scale * pt_scale));
            }
            A.out[A.na++] = inner.back().d;
        }
        A.ptix[A.na - 1][bidx.at(Lv.pts[pi].b)] = (signed char)A.npt;
        A.pt[A.npt++] = Lv.pts[pi].pt.get();
    }
    {
        int ntile = c->N / HE_LT_KT;
        long tiles = (long)L * ntile;
        dim3 grid((unsigned)std::min<long>(tiles, c->max_grid / 4), 1);
        size_t smem = (size_t)A.npt * HE_LT_KT * 8;
        ProfScope ps_(c, "lintrans", 8.0 * c->N * ((double)L * A.npt + (double)x.nct * 2 * L * (A.nb + A.na)));
        if (tune_pick(c, HE_TUNE_LT_ROWS, L, x.nct, 2 * x.nct <= 8)) {   // a few rows: no staging
            if (x.nct == 1 && (A.nb == 4 || A.nb == 8 || A.nb == 16)) {   // both rows' baby steps in registers
                // few limbs (the low SlotToCoeff levels): the giant steps over 2 or 4 threads
                dim3 g1 = grid_for(c, (long)L << c->logN);
                long cta = ((long)L << c->logN) / 256;
                g1.y = cta * 4 <= c->max_grid ? 4 : cta * 2 <= c->max_grid ? 2 : 1;
                if ((int)g1.y > A.na) g1.y = std::max(1, A.na);
                launch_lt_ct1(g1, c->st, A, 2, L, qmap(L), c->d_mods, c->logN);
            }
            else
                klaunch(k_lt_bsgs_direct, grid_for(c, (long)L << c->logN), 256, 0, c->st)(A, 2 * x.nct, L, qmap(L),
                                                                                     c->d_mods, c->logN);
        }
        else
            klaunch(k_lt_bsgs, grid, 256, smem, c->st)(A, 2 * x.nct, L, qmap(L), c->d_mods, c->logN);
    }
    LAUNCH_CHECK();
    // acc = sum_a Rot(out_a, a g hmin): the c0(X^g) parts are added over Q_l, the key-switch
    // inner products of the c1(X^g) parts are summed over Q_l u P and brought down by P once
    DCt acc;
    bool have_acc = false;
    for (size_t i = 0; i < gi.size(); i++)
        if (gi[i] == 0) {
            acc = inner[i];
            have_acc = true;
        }
    if (!have_acc) {
        acc = ct_new(c, x.level, x.nct, x.scale * pt_scale);
        {
            ProfScope ps_(c, "copy", 0);
            CK(cudaMemsetAsync(acc.d, 0, (size_t)acc.nct * acc.cs(c) * 8, c->st));
        }
    }
    DPtr ext;
    bool have_ext = false;
    if (small) {
        // one ModUp of every giant step's c1 (a = 0 included, unused), one launch summing all
        // their key-switch inner products, one ModDown
        int al = c->alpha, nd = (L + al - 1) / al, nl = L + al;
        DPtr dig = ks_modup(c, innerbuf.get() + (long)L * c->N, x.cs(c), (int)gi.size() * x.nct, L);
        KsMulti M{};
        for (size_t i = 0; i < gi.size(); i++) {
            if (gi[i] == 0) continue;
            int ga = galois_for_rot(c, (long)gi[i] * Lv.g * Lv.hmin);
            REQUIRE(M.n < 16, HE_EINVAL, "lintrans: too many giant steps");
            M.key[M.n] = get_key(c, ga);
            M.g[M.n] = ga;
            M.dig_off[M.n] = (long)i * x.nct * nd * nl * c->N;
            M.n++;
            automorph_acc(c, acc, inner[i], ga);
            c->cnt[1]++;
        }
        if (M.n) {
            ext = dalloc(c, (size_t)x.nct * 2 * nl * c->N);
            {
                ProfScope ps(c, "ks_inner", 8.0 * c->N * M.n * ((double)x.nct * nd * nl + 2.0 * nd * nl) +
                                                8.0 * c->N * 2.0 * x.nct * nl);
                klaunch(k_ks_inner_sum, grid_for(c, (long)nl << c->logN), 256, 0, c->st)(
                    ext.get(), dig.get(), x.nct, nd, L, al, extmap(c, L), c->d_mods, c->nm, c->nq, c->logN, M);
            }
            LAUNCH_CHECK();
            c->cnt[0] += (long)M.n * x.nct;
            ks_moddown(c, ext.get(), x.nct, L, acc.d, acc.cs(c), acc.d, acc.cs(c));
        }
        acc.scale = x.scale * pt_scale;
        return rescale(c, acc);
    }
    for (size_t i = 0; i < gi.size(); i++) {
        if (gi[i] == 0) continue;
        int ga = galois_for_rot(c, (long)gi[i] * Lv.g * Lv.hmin);
        const uint64_t *key = get_key(c, ga);
        if (!have_ext) ext = dalloc(c, (size_t)x.nct * 2 * (L + c->alpha) * c->N);
        DPtr dig = ks_modup(c, inner[i].d + (long)L * c->N, inner[i].cs(c), x.nct, L);
        ks_inner_into(c, ext.get(), dig.get(), x.nct, L, ga, key, have_ext);
        automorph_acc(c, acc, inner[i], ga);
        have_ext = true;
        c->cnt[1]++;
    }
    if (have_ext) ks_moddown(c, ext.get(), x.nct, L, acc.d, acc.cs(c), acc.d, acc.cs(c));
    acc.scale = x.scale * pt_scale;
    return rescale(c, acc);
}

static std::vector<int> lt_rotation_steps(he_ctx *c, const LtDesc &lv) {
    int r = lv.nstage, E = (1 << r) - 1, g = bsgs_g(r);
    int hmin = lv.h[0];
    for (int k = 1; k < r; k++) hmin = std::min(hmin, lv.h[k]);
    std::vector<int> out;
    for (int b = 1; b < g; b++) out.push_back(b * hmin);
    for (int a = floordiv(-E, g); a <= floordiv(E, g); a++)
        if (a != 0) out.push_back(a * g * hmin);
    return out;
}

// ------------------------------------------------------------------------- bootstrapping
static DCt bootstrap(he_ctx *c, const DCt &x, double gain, double out_scale) {
    REQUIRE(c->bootstrap, HE_EINVAL, "bootstrapping not enabled");
    REQUIRE(x.level >= c->stc_levels, HE_ELEVEL, "bootstrap: level too low");
    std::unique_ptr<PhaseScope> ph(new PhaseScope(c, "bootstrap.stc"));
    DCt y = ct_drop(c, x, c->stc_levels);
    std::vector<LtDesc> lv = lt_levels(c, c->stc_levels, 0);
    for (int g = 0; g < c->stc_levels; g++) y = lt_eval_level(c, y, lv[g], g == 0 ? gain : 1.0, (double)c->mods[y.level]);
    double d_in = y.scale;
    int top = c->nq - 1;
    ph.reset();   // the previous step's scope ends first (NVTX ranges nest)
    ph.reset(new PhaseScope(c, "bootstrap.modraise"));
    DCt z = mod_raise(c, y, top);
    z.scale = (double)c->mods[0];
    int em_in = top - c->cts_levels;
    double s_em = (double)c->mods[em_in];
    ph.reset();   // the previous step's scope ends first (NVTX ranges nest)
    ph.reset(new PhaseScope(c, "bootstrap.cts"));
    lv = lt_levels(c, c->cts_levels, 1);
    for (int g = 0; g < c->cts_levels; g++) {
        double gn = g == c->cts_levels - 1 ? 1.0 / (2.0 * c->em_K) : 1.0;
        double qs = (double)c->mods[z.level];
        double pts = g == c->cts_levels - 1 ? (qs * s_em) / z.scale : qs;
        z = lt_eval_level(c, z, lv[g], gn, pts);
    }
    ph.reset();   // the previous step's scope ends first (NVTX ranges nest)
    ph.reset(new PhaseScope(c, "bootstrap.evalmod"));
    DCt cj = rotate(c, z, 2 * c->N - 1);
    ct_add_inplace(c, z, cj);
    int lp = c->user_top + c->em_r;
    double s_f = (out_scale * (double)c->mods[0]) / (2.0 * HE_PI * d_in);
    double s_in = s_f;
    for (int i = c->em_r; i >= 1; i--) s_in = sqrt(s_in * (double)c->mods[lp - i + 1]);
    DCt cc = poly_eval(c, z, c->em_c, lp, s_in);
    for (int i = 0; i < c->em_r; i++) {
        DCt sq = hmult(c, cc, cc);
        ct_mul_int(c, sq, 2);
        ct_add_const(c, sq, h_round(-sq.scale));
        cc = sq;
    }
    cc.scale = ((cc.scale * (2.0 * HE_PI)) * d_in) / (double)c->mods[0];
    c->cnt[4]++;
    return cc;
}

// ------------------------------------------------------------------------- Softmax circuit
struct Plan {
    int n, k, exp_deg, method = 0;   // method 0: Alg. 2 + Alg. 3; 1: Alg. 4 (version B)
    double M, boost;
    std::vector<double> exp_c;
    std::vector<int> inv_deg;
    std::vector<std::vector<double>> inv_c;
    std::vector<double> a, b, gs, gl;
    std::vector<double> expo, lam_max, b_max;   // Alg. 4 only
};

static double qd(he_ctx *c, int l) { return (double)c->mods[l]; }

static void affine_to_unit(he_ctx *c, DCt &x, double a, double b) {
    double alpha = 2.0 / (b - a), beta = -(a + b) / (b - a);
    x.scale = x.scale / alpha;
    ct_add_const(c, x, h_round(beta * x.scale));
}

static DCt bts_boosted(he_ctx *c, const Plan &p, const DCt &x, double gain, double out_scale) {
    DCt y = bootstrap(c, x, gain * p.boost, out_scale / p.boost);
    y.scale = y.scale * p.boost;
    return y;
}

// fallback: y too low to feed S = sum y^2 into a bootstrappable level
static bool main_bts(he_ctx *c, const Plan &p, int j, int ly) {
    (void)p;
    (void)j;
    return c->bootstrap && ly < c->bts_min + 1;
}
// z = lam y at product level lz is bootstrapped when another round follows and y = z^2 would
// sit below bts_min + 1; z's maximum lies in [n^{-1/2}, 1] (Sec. 3.2), so its bootstrapping
// error is small relative to the values, unlike y's for flat distributions
static bool z_bts(he_ctx *c, const Plan &p, int j, int lz) {
    return c->bootstrap && j < p.k - 1 && lz - 2 < c->bts_min + 1;
}
static bool s_bts(he_ctx *c, const Plan &p, int j, int ly) {
    return c->bootstrap && ((ly - 1) - ilog2c(p.inv_deg[j] + 1) - 1 < c->bts_min);
}
static double y_target(he_ctx *c, const Plan &p, int j, int ly) {
    double delta = std::ldexp(1.0, c->log_scale);
    if (j >= p.k || main_bts(c, p, j, ly) || s_bts(c, p, j, ly)) return delta;
    double ap = (2.0 / (p.b[j] - p.a[j])) * p.gs[j];
    return sqrt((ap * qd(c, ly - 1)) * qd(c, ly));
}

static DCt rotsum(he_ctx *c, DCt x, int stride, int nrot) {
    for (int i = 0; i < nrot; i++) {
        DCt r = rotate(c, x, galois_for_rot(c, (long)stride << i));
        ct_add_inplace(c, x, r);
    }
    return x;
}

// Diagnostics: with HE_DEBUG_DIR set, the decrypted slots of the first ciphertext of each
// intermediate are written to <dir>/<round>_<name>.bin (N/2 complex doubles).
static void dbg_dump(he_ctx *c, const char *what, int j, const DCt &x) {
    const char *dir = getenv("HE_DEBUG_DIR");
    if (!dir) return;
    std::vector<double2> z = decrypt_slots(c, x, 0);
    char fn[512];
    snprintf(fn, sizeof fn, "%s/%d_%s.bin", dir, j, what);
    FILE *f = fopen(fn, "wb");
    if (!f) return;
    fwrite(z.data(), sizeof(double2), z.size(), f);
    fclose(f);
}

// sum_c y_c (x) y_c (degree 2, [G][3][level+1][N], NTT form, one sum per group): ys holds the m
// main-thread ciphertexts as one batch (or m batches of one); with G > 1 ys[0] holds G groups
static DPtr tensor_sum(he_ctx *c, const std::vector<DCt> &ys, int m, int G) {
    int ly = ys[0].level;
    int L = ly + 1;
    DPtr d = dalloc(c, (size_t)G * 3 * L * c->N);
    PhaseScope ph(c, "main");   // per-ciphertext tensors and their sum
    bool first = true;
    if (G > 1) {
        const DCt &y = ys[0];
        long t3 = 3L * L * c->N;
        DPtr dd = m > 1 ? dalloc(c, (size_t)y.nct * t3) : DPtr();
        tensor_into(c, m > 1 ? dd.get() : d.get(), y, y, ly, false);
        // group g: d[g] = sum_i dd[g m + i] (3 polynomials of L limbs each)
        for (int g = 0; m > 1 && g < G; g++) {
            for (int i = 1; i < m; i++) {
                const uint64_t *acc = i == 1 ? dd.get() + (long)g * m * t3 : d.get() + g * t3;
                {
                    ProfScope ps_(c, "elementwise", 0);
                    klaunch(k_add, grid_for(c, t3), 256, 0, c->st)(d.get() + g * t3, (long)L * c->N, acc, (long)L * c->N,
                                                               dd.get() + ((long)g * m + i) * t3, (long)L * c->N,
                                                               3 * L, L, qmap(L), c->d_mods, c->logN, 0);
                }
                LAUNCH_CHECK();
            }
        }
        first = false;
    }
    for (auto &y : ys) {
        if (G > 1) break;
        if (y.nct == 1) {
            tensor_into(c, d.get(), y, y, ly, !first);
            first = false;
        } else {
            // sum of the per-ciphertext tensors of the batch
            DPtr dd = dalloc(c, (size_t)y.nct * 3 * L * c->N);
            tensor_into(c, dd.get(), y, y, ly, false);
            for (int i = 0; i < y.nct; i++) {
                int cnt = 3 * L;
                long tot = (long)cnt << c->logN;
                if (first && i == 0)
                    {
                        ProfScope ps_(c, "copy", 0);
                        CK(cudaMemcpyAsync(d.get(), dd.get(), (size_t)3 * L * c->N * 8, cudaMemcpyDeviceToDevice, c->st));
                    }
                else {
                    ProfScope ps_(c, "elementwise", 0);
                    klaunch(k_add, grid_for(c, tot), 256, 0, c->st)(d.get(), (long)L * c->N, d.get(), (long)L * c->N,
                                                                dd.get() + (long)i * 3 * L * c->N, (long)L * c->N,
                                                                cnt, L, qmap(L), c->d_mods, c->logN, 0);
                }
                LAUNCH_CHECK();
            }
            first = false;
        }
    }
    return d;
}

// S = Relin(sum_c y_c (x) y_c) rescaled, from the tensor sum d of ciphertexts at `level` and scale ys
static DCt relin_sum(he_ctx *c, const uint64_t *d, int level, int G, double ys) {
    PhaseScope pa(c, "aux");    // one relinearisation of the sum
    DCt S = relin_rescale(c, d, level, G, ys * ys);
    c->cnt[2]++;
    return S;
}

static DCt square_sum(he_ctx *c, const std::vector<DCt> &ys, int m, int G) {
    DPtr d = tensor_sum(c, ys, m, G);
    return relin_sum(c, d.get(), ys[0].level, G, ys[0].scale);
}

// ys: the m main-thread ciphertexts, as one batch (batched) or m batches of one; with G > 1
// (batched only) ys[0] holds G independent groups of m ciphertexts each (G m ciphertexts): the
// sum of squares stays inside each group and the auxiliary thread runs over a batch of G
static std::vector<DCt> softmax_run(he_ctx *c, const Plan &p, std::vector<DCt> ys, int m, int G = 1) {
    REQUIRE(G == 1 || (ys.size() == 1 && ys[0].nct == G * m), HE_EINVAL, "softmax: groups need one batch");
    int n0 = c->n0, n = p.n;
    int stride = (int)((long)m * n0 / n);
    int nrot = ilog2c(n / m);
    int ut = c->user_top;
    double delta = std::ldexp(1.0, c->log_scale);
    {
        PhaseScope ph(c, "main");
        for (auto &y : ys) {
            affine_to_unit(c, y, -p.M, 0.0);
            int lvl = y.level - ilog2c(p.exp_deg + 1);
            y = poly_eval(c, y, p.exp_c, lvl, y_target(c, p, 0, lvl));
        }
    }
    dbg_dump(c, "y0", 0, ys[0]);
    for (int j = 0; j < p.k; j++) {
        int ly = ys[0].level;
        if (main_bts(c, p, j, ly)) {
            double so = y_target(c, p, j, ut);
            for (auto &y : ys) y = bts_boosted(c, p, y, 1.0, so);
            ly = ys[0].level;
            dbg_dump(c, "ybts", j, ys[0]);
        }
        DCt S = square_sum(c, ys, m, G);
        PhaseScope ph_aux(c, "aux");
        S = rotsum(c, S, stride, nrot);
        dbg_dump(c, "S", j, S);
        int dj = ilog2c(p.inv_deg[j] + 1);
        DCt v;
        if (!s_bts(c, p, j, ly)) {
            v = S;
            v.scale = v.scale / p.gs[j];
        } else {
            double so = (2.0 / (p.b[j] - p.a[j])) * qd(c, ut);
            v = bts_boosted(c, p, S, p.gs[j], so);
        }
        dbg_dump(c, "v", j, v);
        affine_to_unit(c, v, p.a[j], p.b[j]);
        int lp = v.level - dj;
        DCt lam = poly_eval(c, v, p.inv_c[j], lp, delta);
        dbg_dump(c, "lam", j, lam);
        // lambda is bootstrapped right after the polynomial when it would end below y
        // (except in the last round if two levels remain); masking and replication follow,
        // so every slot of a Softmax carries the same value and error (Alg. 3, Steps 7-10)
        bool lam_bts = c->bootstrap && lp - 1 < ly && !(j == p.k - 1 && lp - 1 >= 2);
        int llam = lam_bts ? ut - 1 : lp - 1;
        int lz = std::min(llam, ly);
        bool zb = z_bts(c, p, j, lz);
        double slam;
        if (zb) {
            slam = (delta * qd(c, lz)) / ys[0].scale;
        } else {
            double tgt = y_target(c, p, j + 1, lz - 2);
            double sz = sqrt(tgt * qd(c, lz - 1));
            slam = (sz * qd(c, lz)) / ys[0].scale;
        }
        int lm = lp;
        if (lam_bts) {
            lam = bts_boosted(c, p, lam, p.gl[j], delta);
            lm = lam.level;
        }
        std::vector<double2> mk(n0, make_double2(0.0, 0.0));
        double mval = sqrt(p.gs[j]);
        for (int i = 0; i < stride; i++) mk[i].x = mval;
        double smk = (slam * qd(c, lm)) / lam.scale;
        if (lam_bts) smk = smk / p.gl[j];
        char mkey[128];
        snprintf(mkey, sizeof mkey, "mask:%d:%d:%a:%a", stride, lm, mval, smk);
        auto mit = c->pt_cache.find(mkey);
        if (mit == c->pt_cache.end()) {
            mit = c->pt_cache.emplace(mkey, encode(c, mk, smk, lm)).first;
            cache_entry_made(c);
        }
        ct_mul_plain(c, lam, mit->second.get());
        lam.scale = lam.scale * smk;
        lam = rescale(c, lam);
        lam = rotsum(c, lam, stride, nrot);
        if (lam_bts) lam.scale = lam.scale * p.gl[j];
        dbg_dump(c, "lamf", j, lam);
        double soz = zb ? sqrt(y_target(c, p, j + 1, ut - 1) * qd(c, ut)) : 0.0;
        PhaseScope ph_main(c, "main");
        for (auto &y : ys) {
            DCt z = G > 1 && m > 1 ? hmult_grouped(c, lam, y, m) : hmult(c, lam, y);
            if (zb) z = bts_boosted(c, p, z, 1.0, soz);
            y = hmult(c, z, z);
        }
        dbg_dump(c, "y", j, ys[0]);
    }
    return ys;
}

// Alg. 4 (version B, Sec. 4.3) with the auxiliary thread of Alg. 3 on the many-ciphertext
// packing of Sec. 4.2.  lambda_j = S_j^(-1/2^j) with S_j = sum (y^(j-1))^2 (the reading under which
// every round normalises: lambda_1 ... lambda_j applied to y^(0) and squared j times gives y^(j));
// the main thread never bootstraps, the auxiliary ciphertext does (S_j and lambda_j, each alone):
//   u = 2x/M + 1; y0 = P_exp(u) at scale sqrt(Delta q_ly0), so that S_1 lands at Delta
//   for j = 1..k:
//     S_j  = RotSum(relinearised sum_c y_c (x) y_c)      (y = y0 for j = 1, y^(j-1) after)
//     v    = Bootstrap(gain_s S_j) on [a_j, b_j], mapped to [-1, 1]
//     lam  = P_j(v) gain_s^(1/2^j) (gain folded into the coefficients; a polynomial too deep to
//            end above the bootstrapping input level is evaluated split, split_eval)
//     lam  is bootstrapped with gain 1/lam_max_j, then Lam = Lam * lam (Lam = lam for j = 1):
//            one value per Softmax in slots [0, L), one level lower every iteration
//     lr   = RotSum(Lam (.) mask) with the mask 1 on [0, L) encoded at the scale that makes z
//            land where its j squarings need it
//     z_c  = lr * y0_c; y^(j)_c = z_c^(2^j) (j squarings)
// Every free scale is chosen so that the next polynomial input sits at the scale of its level's
// prime and every bootstrapping input at Delta.
static DCt split_eval(he_ctx *c, const Plan &p, const DCt &v, const std::vector<double> &cf, int dj, double delta,
                      double bmax) {
    // p(u) = A(u) + T_h(u) B(u), h = 2^(dj-1), A and B of degree < h (T_h T_i = (T_(h+i) + T_(h-i))/2):
    // A, B and T_(h/2) take dj - 1 levels each; T_(h/2) and B are bootstrapped, T_h = 2 T_(h/2)^2 - 1,
    // and T_h B joins A at the bootstrapping input level
    REQUIRE(bmax > 0, HE_EINVAL, "split polynomial: the plan gives no bound for its upper half");
    int top = v.level, h = 1 << (dj - 1), d = (int)cf.size() - 1;
    std::vector<double> a_c(cf.begin(), cf.begin() + h), b_c(d - h + 1, 0.0);
    b_c[0] = cf[h];
    for (int i = 1; i <= d - h; i++) {
        b_c[i] = 2.0 * cf[h + i];
        a_c[h - i] = a_c[h - i] - cf[h + i];
    }
    int lo = top - (dj - 1);
    std::vector<double> e(h / 2 + 1, 0.0);
    e[h / 2] = 1.0;
    double s_t = sqrt(2.0 * qd(c, top) * delta);
    // the T and B halves are independent one-ciphertext chains (each with a bootstrapping) and
    // run on two side streams, concurrently with each other and with A on the main stream
    DCt th, bb;
    Branch br_t(c, 0), br_b(c, 1);   // both fork here
    br_t.enter();
    {
        DCt t = bts_boosted(c, p, poly_eval(c, v, e, lo, delta), 1.0, s_t);
        th = hmult(c, t, t);                  // t^2 at 2 Delta = 2 t^2 - 1 + 1 at Delta
        th.scale = th.scale / 2.0;
        ct_add_const(c, th, h_round(-1.0 * th.scale));
    }
    br_t.leave();
    br_b.enter();
    bb = bts_boosted(c, p, poly_eval(c, v, b_c, lo, delta), 1.0 / bmax, qd(c, top - 1) * bmax);
    bb.scale = bb.scale / bmax;               // B at scale q_(top-1)
    br_b.leave();
    // A needs only the scale of T_h B, which the host knows from the scale bookkeeping alone
    double prod_scale = (th.scale * bb.scale) / qd(c, std::min(th.level, bb.level));
    DCt a = poly_eval(c, v, a_c, lo, prod_scale);
    br_t.join();
    br_b.join();
    DCt prod = hmult(c, th, bb);
    REQUIRE(prod.scale == prod_scale, HE_EINVAL, "split polynomial: scale bookkeeping");
    DCt out = ct_drop(c, prod, lo);
    ct_add_inplace(c, out, a);
    return out;
}

// the mask (value mval on slots [0, stride), 0 elsewhere) encoded at `scale` for `level`,
// once per (stride, level, value, scale)
static const uint64_t *mask_pt(he_ctx *c, int stride, int level, double mval, double scale) {
    char mkey[128];
    snprintf(mkey, sizeof mkey, "mask:%d:%d:%a:%a", stride, level, mval, scale);
    auto mit = c->pt_cache.find(mkey);
    if (mit == c->pt_cache.end()) {
        std::vector<double2> mk(c->n0, make_double2(0.0, 0.0));
        for (int i = 0; i < stride; i++) mk[i].x = mval;
        mit = c->pt_cache.emplace(mkey, encode(c, mk, scale, level)).first;
        cache_entry_made(c);
    }
    return mit->second.get();
}

// Alg. 4, main thread before the rounds: u = 2x/M + 1, y0 = P_exp(u) at level ly0 with scale
// sqrt(Delta q_ly0), so that S_1 = sum y0^2 lands at Delta
static int alg4_ly0(he_ctx *c, const Plan &p, int level_in) { return level_in - ilog2c(p.exp_deg + 1); }

static void alg4_exp(he_ctx *c, const Plan &p, std::vector<DCt> &ys) {
    PhaseScope ph(c, "main");
    double delta = std::ldexp(1.0, c->log_scale);
    int ly0 = alg4_ly0(c, p, ys[0].level);
    for (auto &y : ys) {
        affine_to_unit(c, y, -p.M, 0.0);
        y = poly_eval(c, y, p.exp_c, ly0, sqrt(delta * qd(c, ly0)));
    }
}

// Alg. 4, auxiliary thread of round j (1-based), from the relinearised sum of squares S (G groups,
// before the rotate-and-sum) of the m main-thread ciphertexts per group: returns lr, the
// replicated (mask, rotate-and-sum) product of Lambda = lambda_1 ... lambda_j, and updates lam_c
// (Lambda; have_lam false before round 1).  y0_scale: the scale of y0; ly0: its level.
static DCt alg4_aux(he_ctx *c, const Plan &p, int j, DCt S, int m, int ly0, double y0_scale, DCt &lam_c,
                    bool &have_lam) {
    PhaseScope ph_aux(c, "aux");
    const int jj = j - 1;   // plan index
    int n0 = c->n0, stride = (int)((long)m * n0 / p.n), nrot = ilog2c(p.n / m), top = c->user_top;
    double delta = std::ldexp(1.0, c->log_scale);
    S = rotsum(c, S, stride, nrot);
    double a = p.a[jj], b = p.b[jj];
    DCt v = bts_boosted(c, p, S, p.gs[jj], (2.0 / (b - a)) * qd(c, top));
    affine_to_unit(c, v, a, b);
    std::vector<double> cf = p.inv_c[jj];
    double g = pow(p.gs[jj], p.expo[jj]);
    for (auto &x : cf) x = x * g;
    int dj = ilog2c((int)cf.size());
    int lp = top - dj;
    DCt lam = lp < c->bts_min ? split_eval(c, p, v, cf, dj, delta, p.b_max[jj]) : poly_eval(c, v, cf, lp, delta);
    double lmax = p.lam_max[jj];
    int lam_lv = have_lam ? lam_c.level : top;
    DCt lb = bts_boosted(c, p, lam, 1.0 / lmax, qd(c, lam_lv) * lmax);
    lb.scale = lb.scale / lmax;           // lambda_j at scale q_(lam_lv)
    lam_c = have_lam ? hmult(c, lam_c, lb) : lb;
    have_lam = true;
    // where z lands and the scale it needs there: j squarings, then (j < k) one more for S
    int lz = ly0 - 1;
    double sz = delta;
    for (int i = (j == p.k ? j : j + 1); i >= 1; i--) sz = sqrt(sz * qd(c, lz - i + 1));
    double s_lr = (sz * qd(c, ly0)) / y0_scale;
    double sm = (s_lr * qd(c, lam_c.level)) / lam_c.scale;
    DCt lr = ct_copy(c, lam_c);
    ct_mul_plain(c, lr, mask_pt(c, stride, lam_c.level, 1.0, sm));
    lr.scale = lr.scale * sm;
    return rotsum(c, rescale(c, lr), stride, nrot);
}

// Alg. 4, main thread of round j: y^(j)_c = (lr y0_c)^(2^j) (j squarings)
static void alg4_update(he_ctx *c, int j, const DCt &lr, const std::vector<DCt> &y0, std::vector<DCt> &ys, int m, int G) {
    PhaseScope ph_main(c, "main");
    for (size_t i = 0; i < ys.size(); i++) {
        DCt z = G > 1 && m > 1 ? hmult_grouped(c, lr, y0[i], m) : hmult(c, lr, y0[i]);
        for (int t = 0; t < j; t++) z = hmult(c, z, z);
        ys[i] = z;
    }
}

static std::vector<DCt> softmax_run_b(he_ctx *c, const Plan &p, std::vector<DCt> ys, int m, int G = 1) {
    REQUIRE(G == 1 || (ys.size() == 1 && ys[0].nct == G * m), HE_EINVAL, "softmax: groups need one batch");
    REQUIRE(c->bootstrap, HE_EINVAL, "Alg. 4 needs bootstrapping");
    alg4_exp(c, p, ys);
    const std::vector<DCt> y0 = ys;
    const int ly0 = y0[0].level;
    DCt lam_c;
    bool have_lam = false;
    for (int j = 1; j <= p.k; j++) {
        DCt S = square_sum(c, ys, m, G);
        DCt lr = alg4_aux(c, p, j, S, m, ly0, y0[0].scale, lam_c, have_lam);
        alg4_update(c, j, lr, y0, ys, m, G);
    }
    return ys;
}

// ------------------------------------------------------------------------- context creation
static void build_tables(he_ctx *c) {
    int N = c->N, nm = c->nm;
    c->modc.resize(nm);
    for (int i = 0; i < nm; i++) {
        uint64_t q = c->mods[i];
        int s = 64 - __builtin_clzll(q);
        REQUIRE(s <= 60 && s >= 20, HE_EINVAL, "modulus size");   // 16q < 2^64 in the NTT
        REQUIRE((q - 1) % (2 * (uint64_t)N) == 0, HE_EINVAL, "modulus not 1 mod 2N");
        ModC m;
        m.q = q;
        m.s = s;
        m.pad = 0;
        m.mu = (uint64_t)(((u128)1 << (s + 63)) / q);
        uint64_t inv = q;                          // q^{-1} mod 2^64 by Newton's iteration
        for (int it = 0; it < 6; it++) inv *= 2 - q * inv;
        m.qinv = 0 - inv;
        c->modc[i] = m;
    }
    CK(cudaMalloc(&c->d_mods, sizeof(ModC) * nm));
    CK(cudaMemcpy(c->d_mods, c->modc.data(), sizeof(ModC) * nm, cudaMemcpyHostToDevice));
    // NTT tables: psi^{brv(k)} and psi^{-brv(k)} with Shoup companions
    std::vector<uint64_t> tw((size_t)nm * 4 * N), ninv(2 * nm);
    for (int t = 0; t < nm; t++) {
        uint64_t q = c->mods[t], psi = h_root(q, N);
        REQUIRE(psi, HE_EINVAL, "no 2N-th root");
        uint64_t ipsi = h_inv(psi, q);
        std::vector<uint64_t> pw(N), ipw(N);
        pw[0] = ipw[0] = 1;
        for (int i = 1; i < N; i++) {
            pw[i] = h_mulmod(pw[i - 1], psi, q);
            ipw[i] = h_mulmod(ipw[i - 1], ipsi, q);
        }
        uint64_t *T = tw.data() + (size_t)t * 4 * N;
        for (int k = 0; k < N; k++) {
            int r = 0;
            for (int b = 0; b < c->logN; b++) r |= ((k >> b) & 1) << (c->logN - 1 - b);
            T[k] = pw[r];
            T[N + k] = h_shoup(pw[r], q);
            T[2 * N + k] = ipw[r];
            T[3 * N + k] = h_shoup(ipw[r], q);
        }
        uint64_t ni = h_inv((uint64_t)N % q, q);
        ninv[2 * t] = ni;
        ninv[2 * t + 1] = h_shoup(ni, q);
    }
    {
        std::vector<ulonglong2> tw2((size_t)nm * 2 * N);
        for (int t = 0; t < nm; t++) {
            const uint64_t *T = tw.data() + (size_t)t * 4 * N;
            for (int k = 0; k < N; k++) {
                tw2[(size_t)t * 2 * N + k] = make_ulonglong2(T[k], T[N + k]);
                tw2[(size_t)t * 2 * N + N + k] = make_ulonglong2(T[2 * N + k], T[3 * N + k]);
            }
        }
        CK(cudaMalloc(&c->d_tw2, tw2.size() * sizeof(ulonglong2)));
        CK(cudaMemcpy(c->d_tw2, tw2.data(), tw2.size() * sizeof(ulonglong2), cudaMemcpyHostToDevice));
    }
    CK(cudaMalloc(&c->d_ninv, ninv.size() * 8));
    CK(cudaMemcpy(c->d_ninv, ninv.data(), ninv.size() * 8, cudaMemcpyHostToDevice));
    // ModUp constants per (level, digit)
    int al = c->alpha;
    std::vector<uint64_t> cv;
    c->cv_off.assign(c->nq, {});
    for (int Lm1 = 0; Lm1 < c->nq; Lm1++) {
        int L = Lm1 + 1, nl = L + al, nd = (L + al - 1) / al;
        for (int j = 0; j < nd; j++) {
            int lo = j * al, hi = std::min(L, lo + al), ds = hi - lo;
            c->cv_off[Lm1].push_back(cv.size());
            std::vector<uint64_t> qhinv(ds), qhinvs(ds), qh((size_t)ds * nl);
            for (int i = lo; i < hi; i++) {
                uint64_t qi = c->mods[i], prod = 1 % qi;
                for (int i2 = lo; i2 < hi; i2++)
                    if (i2 != i) prod = h_mulmod(prod, c->mods[i2] % qi, qi);
                qhinv[i - lo] = h_inv(prod, qi);
                qhinvs[i - lo] = h_shoup(qhinv[i - lo], qi);
                for (int t = 0; t < nl; t++) {
                    uint64_t mt = c->mods[t < L ? t : c->nq + (t - L)], pr = 1 % mt;
                    for (int i2 = lo; i2 < hi; i2++)
                        if (i2 != i) pr = h_mulmod(pr, c->mods[i2] % mt, mt);
                    qh[(size_t)(i - lo) * nl + t] = h_mont(pr, mt);
                }
            }
            cv.insert(cv.end(), qhinv.begin(), qhinv.end());
            cv.insert(cv.end(), qhinvs.begin(), qhinvs.end());
            cv.insert(cv.end(), qh.begin(), qh.end());
        }
    }
    CK(cudaMalloc(&c->d_cv, cv.size() * 8));
    CK(cudaMemcpy(c->d_cv, cv.data(), cv.size() * 8, cudaMemcpyHostToDevice));
    // ModDown constants
    std::vector<uint64_t> md(2 * al + (size_t)al * c->nq), pinv(2 * c->nq);
    std::vector<int> pidx(al);
    for (int k = 0; k < al; k++) {
        uint64_t pk = c->mods[c->nq + k], prod = 1 % pk;
        for (int k2 = 0; k2 < al; k2++)
            if (k2 != k) prod = h_mulmod(prod, c->mods[c->nq + k2] % pk, pk);
        md[k] = h_inv(prod, pk);
        md[al + k] = h_shoup(md[k], pk);
        pidx[k] = c->nq + k;
        for (int i = 0; i < c->nq; i++) {
            uint64_t q = c->mods[i], pr = 1 % q;
            for (int k2 = 0; k2 < al; k2++)
                if (k2 != k) pr = h_mulmod(pr, c->mods[c->nq + k2] % q, q);
            md[2 * al + (size_t)k * c->nq + i] = h_mont(pr, q);
        }
    }
    for (int i = 0; i < c->nq; i++) {
        uint64_t q = c->mods[i], pm = 1 % q;
        for (int k = 0; k < al; k++) pm = h_mulmod(pm, c->mods[c->nq + k] % q, q);
        pinv[2 * i] = h_inv(pm, q);
        pinv[2 * i + 1] = h_shoup(pinv[2 * i], q);
    }
    CK(cudaMalloc(&c->d_mdcv, md.size() * 8));
    CK(cudaMemcpy(c->d_mdcv, md.data(), md.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMalloc(&c->d_pinv, pinv.size() * 8));
    CK(cudaMemcpy(c->d_pinv, pinv.data(), pinv.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMalloc(&c->d_pidx, pidx.size() * sizeof(int)));
    CK(cudaMemcpy(c->d_pidx, pidx.data(), pidx.size() * sizeof(int), cudaMemcpyHostToDevice));
    // inverse-transform scale factors N^{-1} f mod p (with Shoup companions) where f is the first
    // factor [qhat^{-1}] of the basis conversion that reads the transform's output
    auto fold = [&](std::vector<uint64_t> &tab, size_t row, int p, uint64_t f) {
        uint64_t q = c->mods[p], v = h_mulmod(ninv[2 * p], f % q, q);
        tab[row * 2 * nm + 2 * p] = v;
        tab[row * 2 * nm + 2 * p + 1] = h_shoup(v, q);
    };
    {
        std::vector<uint64_t> up((size_t)c->nq * 2 * nm, 0), down((size_t)2 * nm, 0);
        for (int Lm1 = 0; Lm1 < c->nq; Lm1++) {
            int L = Lm1 + 1;
            for (int j = 0; j * al < L; j++) {
                int lo = j * al, ds = std::min(al, L - lo);
                for (int i = 0; i < ds; i++) fold(up, Lm1, lo + i, cv[c->cv_off[Lm1][j] + i]);   // qhinv
            }
        }
        for (int k = 0; k < al; k++) fold(down, 0, c->nq + k, md[k]);   // phinv
        CK(cudaMalloc(&c->d_ninv_up, up.size() * 8));
        CK(cudaMemcpy(c->d_ninv_up, up.data(), up.size() * 8, cudaMemcpyHostToDevice));
        CK(cudaMalloc(&c->d_ninv_down, down.size() * 8));
        CK(cudaMemcpy(c->d_ninv_down, down.data(), down.size() * 8, cudaMemcpyHostToDevice));
    }
    // rescale constants: q_l^{-1} mod q_i (i < l)
    std::vector<uint64_t> ql((size_t)c->nq * 2 * c->nq, 0);
    for (int l = 1; l < c->nq; l++)
        for (int i = 0; i < l; i++) {
            uint64_t q = c->mods[i], v = h_inv(c->mods[l] % q, q);
            ql[(size_t)l * 2 * c->nq + 2 * i] = v;
            ql[(size_t)l * 2 * c->nq + 2 * i + 1] = h_shoup(v, q);
        }
    CK(cudaMalloc(&c->d_qlinv, ql.size() * 8));
    CK(cudaMemcpy(c->d_qlinv, ql.data(), ql.size() * 8, cudaMemcpyHostToDevice));
    {
        // relinearisation + rescale: D = {q_l, p_0 .. p_{alpha-1}}
        int nd = al + 1;
        c->rrcv_stride = 2 * (size_t)nd + (size_t)nd * c->nq;
        std::vector<uint64_t> rrcv((size_t)c->nq * c->rrcv_stride, 0), rrpq((size_t)c->nq * 4 * c->nq, 0);
        std::vector<int> rridx((size_t)c->nq * nd, 0);
        for (int l = 1; l < c->nq; l++) {
            uint64_t md[HE_MAX_LIMBS];
            int mi[HE_MAX_LIMBS];
            md[0] = c->mods[l];
            mi[0] = l;
            for (int k = 0; k < al; k++) {
                md[1 + k] = c->mods[c->nq + k];
                mi[1 + k] = c->nq + k;
            }
            uint64_t *cv = rrcv.data() + (size_t)l * c->rrcv_stride;
            for (int j = 0; j < nd; j++) {
                rridx[(size_t)l * nd + j] = mi[j];
                uint64_t prod = 1 % md[j];
                for (int j2 = 0; j2 < nd; j2++)
                    if (j2 != j) prod = h_mulmod(prod, md[j2] % md[j], md[j]);
                cv[j] = h_inv(prod, md[j]);
                cv[nd + j] = h_shoup(cv[j], md[j]);
                for (int i = 0; i < c->nq; i++) {
                    uint64_t q = c->mods[i], pr = 1 % q;
                    for (int j2 = 0; j2 < nd; j2++)
                        if (j2 != j) pr = h_mulmod(pr, md[j2] % q, q);
                    cv[2 * nd + (size_t)j * c->nq + i] = h_mont(pr, q);
                }
            }
            for (int i = 0; i < l; i++) {
                uint64_t q = c->mods[i], pm = 1 % q;
                for (int k = 0; k < al; k++) pm = h_mulmod(pm, c->mods[c->nq + k] % q, q);
                uint64_t w = h_inv(h_mulmod(pm, c->mods[l] % q, q), q);
                uint64_t *e = rrpq.data() + ((size_t)l * c->nq + i) * 4;
                e[0] = pm;
                e[1] = h_shoup(pm, q);
                e[2] = w;
                e[3] = h_shoup(w, q);
            }
        }
        CK(cudaMalloc(&c->d_rrcv, rrcv.size() * 8));
        CK(cudaMemcpy(c->d_rrcv, rrcv.data(), rrcv.size() * 8, cudaMemcpyHostToDevice));
        CK(cudaMalloc(&c->d_rrpq, rrpq.size() * 8));
        CK(cudaMemcpy(c->d_rrpq, rrpq.data(), rrpq.size() * 8, cudaMemcpyHostToDevice));
        CK(cudaMalloc(&c->d_rridx, rridx.size() * sizeof(int)));
        CK(cudaMemcpy(c->d_rridx, rridx.data(), rridx.size() * sizeof(int), cudaMemcpyHostToDevice));
        std::vector<uint64_t> rr((size_t)c->nq * 2 * nm, 0);
        for (int l = 1; l < c->nq; l++)
            for (int j = 0; j < nd; j++) fold(rr, l, rridx[(size_t)l * nd + j], rrcv[(size_t)l * c->rrcv_stride + j]);
        CK(cudaMalloc(&c->d_ninv_rr, rr.size() * 8));
        CK(cudaMemcpy(c->d_ninv_rr, rr.data(), rr.size() * 8, cudaMemcpyHostToDevice));
    }
    // canonical embedding tables: zeta^j = exp(2 pi i j / 2N), 5^j mod 2N
    int m = 2 * N;
    c->zeta.resize(m);
    for (int j = 0; j < m; j++) {
        double ang = (2.0 * HE_PI * (double)j) / (double)m;
        c->zeta[j] = make_double2(cos(ang), sin(ang));
    }
    c->rg.resize(c->n0);
    long g = 1;
    for (int j = 0; j < c->n0; j++) {
        c->rg[j] = (int)g;
        g = (g * 5) % m;
    }
    CK(cudaMalloc(&c->d_zeta, sizeof(double2) * m));
    CK(cudaMemcpy(c->d_zeta, c->zeta.data(), sizeof(double2) * m, cudaMemcpyHostToDevice));
    CK(cudaMalloc(&c->d_rg, sizeof(int) * c->n0));
    CK(cudaMemcpy(c->d_rg, c->rg.data(), sizeof(int) * c->n0, cudaMemcpyHostToDevice));
    // Gaussian cumulative table: rho(k) = exp(-k^2 / (2 sigma^2)), k <= ceil(6 sigma)
    int kmax = (int)ceil(6.0 * c->sigma);
    double s2 = 2.0 * c->sigma * c->sigma;
    double zsum = exp(-0.0 / s2);
    for (int k = 1; k <= kmax; k++) zsum += 2.0 * exp(-(double)(k * k) / s2);
    std::vector<uint64_t> cdt(kmax);
    double acc = 0.0;
    for (int k = 0; k < kmax; k++) {
        double pk = (k == 0 ? exp(-0.0 / s2) : 2.0 * exp(-(double)(k * k) / s2)) / zsum;
        acc += pk;
        cdt[k] = (uint64_t)(acc * 9223372036854775808.0);
    }
    c->cdt_len = kmax;
    CK(cudaMalloc(&c->d_cdt, sizeof(uint64_t) * kmax));
    CK(cudaMemcpy(c->d_cdt, cdt.data(), sizeof(uint64_t) * kmax, cudaMemcpyHostToDevice));
    // Garner constants for decoding
    REQUIRE(c->nq <= HE_MAX_LIMBS, HE_EINVAL, "too many primes");
    std::vector<uint64_t> radix((size_t)c->nq * HE_MAX_LIMBS, 0), radinv(c->nq);
    std::vector<double> qdv(c->nq);
    for (int i = 0; i < c->nq; i++) {
        uint64_t q = c->mods[i], r = 1 % q;
        for (int j = 0; j < i; j++) {
            radix[(size_t)i * HE_MAX_LIMBS + j] = r;
            r = h_mulmod(r, c->mods[j] % q, q);
        }
        radinv[i] = h_inv(r, q);
        qdv[i] = (double)c->mods[i];
    }
    CK(cudaMalloc(&c->d_radix, radix.size() * 8));
    CK(cudaMemcpy(c->d_radix, radix.data(), radix.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMalloc(&c->d_radinv, radinv.size() * 8));
    CK(cudaMemcpy(c->d_radinv, radinv.data(), radinv.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMalloc(&c->d_qd, qdv.size() * 8));
    CK(cudaMemcpy(c->d_qd, qdv.data(), qdv.size() * 8, cudaMemcpyHostToDevice));
    c->ndig_top = (c->nq + al - 1) / al;
    // the conversion and inner-product kernels hold alpha residues and ndig key words per
    // thread, and their 128-bit sums must stay below q 2^64
    REQUIRE(al >= 1 && al <= 8 && c->ndig_top <= 8, HE_EINVAL, "alpha and the digit count must be at most 8");
    // linear-transform inner sums: up to HE_LT_MAXPT staged plaintext tiles of HE_LT_KT words
    CK(cudaFuncSetAttribute(k_lt_bsgs, cudaFuncAttributeMaxDynamicSharedMemorySize, HE_LT_MAXPT * HE_LT_KT * 8));
    if (c->logN == 16) REQUIRE(ntt_1pass_setup() == 0, HE_EINVAL, "one-pass transform: shared memory limit");
}

// ---- autotuner
// one warm-up run of fn, then the best of reps runs, timed with CUDA events on the context stream
template <class F>
static float time_best(he_ctx *c, int reps, F fn) {
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    fn();
    float best = 1e30f;
    for (int r = 0; r < reps; r++) {
        CK(cudaEventRecord(a, c->st));
        fn();
        CK(cudaEventRecord(b, c->st));
        CK(cudaEventSynchronize(b));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, a, b));
        best = std::min(best, ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

// times variants 0 and 1 of op (forced) with fn and keeps the faster one for (op, L, nct)
template <class F>
static void tune_op(he_ctx *c, int op, int L, int nct, int reps, F fn) {
    he_ctx::TuneRec r;
    const int prev = c->tune_force[op];
    for (int v = 0; v < 2; v++) {
        c->tune_force[op] = v;
        try {
            r.ms[v] = time_best(c, reps, fn);
        } catch (...) {
            c->tune_force[op] = prev;
            throw;
        }
    }
    c->tune_force[op] = prev;
    r.choice = r.ms[1] < r.ms[0] ? 1 : 0;
    c->tune[std::make_tuple(op, L, nct)] = r;
}

static void autotune(he_ctx *c, const std::vector<int> &levels, const std::vector<int> &ncts, int reps) {
    REQUIRE(c->have_keys, HE_ENOKEY, "autotune: keygen first");
    long cnt0[5], l0 = c->launches;
    for (int i = 0; i < 5; i++) cnt0[i] = c->cnt[i];
    std::vector<std::string> cached;
    for (auto &kv : c->lt_cache) cached.push_back(kv.first);
    for (int lv : levels) {
        for (int nct : ncts) {
            int L = lv + 1;
            DCt x = ct_new(c, lv, nct, 1.0);
            {
                ProfScope ps_(c, "keygen", 0);
                klaunch(k_sample_uniform, grid_for(c, (long)2 * nct * L << c->logN), 256, 0, c->st)(
                    x.d, (long)L * c->N, 2 * nct * L, L, qmap(L), c->d_mods, 0x5eedULL + lv, 0x70e0ULL, c->logN);
            }
            LAUNCH_CHECK();
            tune_op(c, HE_TUNE_MODUP, L, nct, reps, [&] { DPtr d = ks_modup(c, x.d + (long)L * c->N, x.cs(c), nct, L); });
            // fused or separate basis conversions: one relinearisation (ModUp, inner product, ModDown)
            tune_op(c, HE_TUNE_FUSE_CONV, L, nct, reps, [&] {
                DCt y = ct_new(c, lv, nct, 1.0);
                DPtr dig = ks_modup(c, x.d + (long)L * c->N, x.cs(c), nct, L);
                ks_finish(c, dig.get(), nct, L, 0, get_key(c, 0), y.d, y.cs(c), nullptr, 0);
            });
            if (!c->bootstrap) continue;
            // the bootstrapping linear-transform level that runs at this level, if any:
            // SlotToCoeff level g at stc_levels - g, CoeffToSlot level g at the top - g
            for (int inverse = 0; inverse < 2; inverse++) {
                int nlev = inverse ? c->cts_levels : c->stc_levels;
                int g = inverse ? (c->nq - 1) - lv : c->stc_levels - lv;
                if (g < 0 || g >= nlev) continue;
                LtDesc d = lt_levels(c, nlev, inverse)[g];
                const LtLevel &Lv = lt_prepare(c, d, 1.0, qd(c, lv), lv);
                std::vector<int> gal;
                for (int b : Lv.baby)
                    if (b != 0) gal.push_back(galois_for_rot(c, (long)b * Lv.hmin));
                if (gal.size() >= 2 && gal.size() <= 16)
                    tune_op(c, HE_TUNE_ROT, L, nct, reps, [&] { std::vector<DCt> r = rotate_hoisted(c, x, gal); });
                tune_op(c, HE_TUNE_LT_ROWS, L, nct, reps, [&] { DCt r = lt_eval_level(c, x, d, 1.0, qd(c, lv)); });
                tune_op(c, HE_TUNE_LT_SMALL, L, nct, reps, [&] { DCt r = lt_eval_level(c, x, d, 1.0, qd(c, lv)); });
            }
        }
    }
    // transforms: 64- against 256-thread CTAs, per direction, over a ladder of limb counts; a
    // launch then takes the choice of the largest ladder count at or below its own
    {
        const int counts[] = {1, 2, 4, 6, 8, 10, 12, 16, 20, 25, 32, 40, 50, 64, 100, 128, 256, 512, 1024, 2048};
        const int maxc = 2048;
        DPtr buf = dalloc(c, (size_t)maxc * c->N);
        {
            ProfScope ps_(c, "keygen", 0);
            klaunch(k_sample_uniform, grid_for(c, (long)maxc << c->logN), 256, 0, c->st)(
                buf.get(), 0, maxc, 1, qmap(1), c->d_mods, 0x5eedULL, 0x70e1ULL, c->logN);
        }
        LAUNCH_CHECK();
        for (int inv = 0; inv < 2; inv++) {
            std::vector<std::pair<int, int>> ladder;
            for (int n : counts) {
                tune_op(c, HE_TUNE_NTT_SMALL, n, inv, reps,
                        [&] { ntt(c, buf.get(), n, qmap(1), c->N, inv != 0); });
                ladder.push_back({n, c->tune[std::make_tuple(HE_TUNE_NTT_SMALL, n, inv)].choice});
            }
            c->ntt_small[inv] = ladder;
        }
        // one pass per limb (N = 2^16) against the two passes with the CTA size just chosen
        if (c->logN == 16)
            for (int inv = 0; inv < 2; inv++) {
                std::vector<std::pair<int, int>> ladder;
                for (int n : counts) {
                    tune_op(c, HE_TUNE_NTT_1PASS, n, inv, reps,
                            [&] { ntt(c, buf.get(), n, qmap(1), c->N, inv != 0); });
                    ladder.push_back({n, c->tune[std::make_tuple(HE_TUNE_NTT_1PASS, n, inv)].choice});
                }
                c->ntt_1pass[inv] = ladder;
            }
    }
    CK(cudaStreamSynchronize(c->st));
    // the tuner's own work is not counted, and its diagonal encodings are dropped
    for (auto it = c->lt_cache.begin(); it != c->lt_cache.end();) {
        if (std::find(cached.begin(), cached.end(), it->first) == cached.end()) it = c->lt_cache.erase(it);
        else ++it;
    }
    for (int i = 0; i < 5; i++) c->cnt[i] = cnt0[i];
    c->launches = l0;
}

// ------------------------------------------------------------------------- C ABI
#define API_BEGIN try {
#define API_END                                      \
    }                                                \
    catch (const HeErr &e) {                         \
        ctx->err = e.msg;                            \
        return e.code;                               \
    }                                                \
    catch (const std::exception &e) {                \
        ctx->err = e.what();                         \
        return HE_EINVAL;                            \
    }                                                \
    return HE_OK;

extern "C" {

int he_context_create(const he_params *p, void *cuda_stream, he_ctx **out) {
    if (!p || !out) return HE_EINVAL;
    *out = nullptr;
    // ring degree: the register-blocked NTT passes exist for N = 2^12 and N = 2^16
    if ((p->log_n != 12 && p->log_n != 16) || p->n_q < 1 || p->n_p < 1 || p->n_q + p->n_p > HE_MAX_MODS ||
        p->n_q > HE_MAX_LIMBS - p->n_p || !p->q || !p->p || p->h < 1 || p->h > (1 << p->log_n))
        return HE_EINVAL;
    he_ctx *c = new he_ctx();
    c->logN = p->log_n;
    c->N = 1 << p->log_n;
    c->n0 = c->N / 2;
    c->nq = p->n_q;
    c->np = p->n_p;
    c->alpha = p->n_p;
    c->nm = c->nq + c->np;
    c->h = p->h;
    c->sigma = p->sigma;
    c->log_scale = p->log_scale;
    c->user_top = p->user_top_level;
    c->bootstrap = p->bootstrap;
    c->stc_levels = p->stc_levels;
    c->cts_levels = p->cts_levels;
    c->bts_min = p->bts_min_level;
    c->em_K = p->em_K;
    c->em_r = p->em_r;
    c->em_deg = p->em_deg;
    if (p->bootstrap && p->em_coeffs) c->em_c.assign(p->em_coeffs, p->em_coeffs + p->em_deg + 1);
    c->st = (cudaStream_t)cuda_stream;
    for (int i = 0; i < p->n_q; i++) c->mods.push_back(p->q[i]);
    for (int i = 0; i < p->n_p; i++) c->mods.push_back(p->p[i]);
    try {
        if (p->bootstrap) {
            REQUIRE(p->em_coeffs && p->em_deg >= 1, HE_EINVAL, "EvalMod coefficients missing");
            REQUIRE(p->user_top_level + p->em_r + ilog2c(p->em_deg + 1) + p->cts_levels == p->n_q - 1, HE_EINVAL,
                    "level map: user_top + EvalMod + CtS levels must reach the top");
        }
        REQUIRE(p->user_top_level < p->n_q, HE_EINVAL, "user_top_level");
        int dev = 0;
        CK(cudaGetDevice(&dev));
        int nsm = 0;
        CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        c->max_grid = nsm * 16;
        build_tables(c);
        // host code must not use the array's name as a device address: look it up once for
        // this device (the current one) and keep it with the context
        CK(cudaGetSymbolAddress((void **)&c->noalloc_scratch, g_rescale_scratch));
    } catch (const HeErr &e) {
        fprintf(stderr, "he_context_create: %s\n", e.msg.c_str());
        he_context_destroy(c);   // frees whatever build_tables allocated before the failure
        return e.code;
    }
    *out = c;
    return HE_OK;
}

void he_context_destroy(he_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->st);
    if (c->gstream) cudaStreamSynchronize(c->gstream);
    for (auto &kv : c->graphs) {
        cudaGraphExecDestroy(kv.second.exec);
        for (auto &r : kv.second.prof) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
    }
    c->graphs.clear();
    if (c->gstream) {
        cudaStreamDestroy(c->gstream);
        cudaEventDestroy(c->gev_in);
        cudaEventDestroy(c->gev_out);
    }
    c->pt_cache.clear();
    c->lt_cache.clear();
    for (int i = 0; i < he_ctx::NSIDE; i++)
        if (c->side[i]) {
            cudaStreamSynchronize(c->side[i]);
            cudaStreamDestroy(c->side[i]);
            cudaEventDestroy(c->fork_ev[i]);
            cudaEventDestroy(c->join_ev[i]);
        }
    for (auto &kv : c->keys) cudaFree(kv.second);
    for (auto &e : c->prof_ev) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    void *ptrs[] = {c->d_mods, c->d_tw2, c->d_ninv, c->d_cv, c->d_mdcv, c->d_pinv, c->d_qlinv, c->d_pidx,
                    c->d_rrcv, c->d_rrpq, c->d_rridx, c->d_ninv_up, c->d_ninv_down, c->d_ninv_rr, c->d_zeta,
                    c->d_rg, c->d_cdt, c->d_radix, c->d_radinv, c->d_qd, c->d_s, c->d_pk};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    delete c;
}

const char *he_last_error(const he_ctx *c) { return c ? c->err.c_str() : "null context"; }
int he_ring_degree(const he_ctx *c) { return c ? c->N : 0; }

// The paper's parameter set (Sec. 5.1.1, the parameter table): N = 2^16, log2(QP) = 1555 and a
// sparse ternary secret of Hamming weight h = 192 give 128-bit security.  Anything with a
// smaller ring, a larger modulus for its ring (the bound taken as proportional to N) or a
// sparser secret is flagged: the small test chains are.
int he_params_insecure(const he_params *p) {
    if (!p || p->log_n < 1 || p->log_n > 20 || p->n_q < 1 || !p->q || p->n_p < 0 || (p->n_p > 0 && !p->p))
        return HE_EINVAL;
    double log_qp = 0.0;
    for (int i = 0; i < p->n_q; i++) log_qp += std::log2((double)p->q[i]);
    for (int i = 0; i < p->n_p; i++) log_qp += std::log2((double)p->p[i]);
    const double bound = 1555.0 * std::ldexp(1.0, p->log_n - 16) + 0.5;
    return (p->log_n < 16 || p->h < 192 || log_qp > bound) ? 1 : 0;
}

// Drops every evaluation key and every captured Softmax graph (whose kernels read those keys):
// a new secret makes all of them stale.  Encoded plaintexts (diagonals, masks) do not depend on
// the secret and stay.
static void drop_keys(he_ctx *c) {
    CK(cudaStreamSynchronize(c->st));
    if (c->gstream) CK(cudaStreamSynchronize(c->gstream));
    for (auto &kv : c->graphs) {
        cudaGraphExecDestroy(kv.second.exec);
        for (auto &r : kv.second.prof) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
    }
    c->graphs.clear();
    for (auto &kv : c->keys) cudaFree(kv.second);
    c->keys.clear();
}

int he_keygen(he_ctx *ctx, uint64_t seed, const int *rot_steps, int n_rot) {
    if (!ctx || n_rot < 0 || (n_rot > 0 && !rot_steps)) return HE_EINVAL;
    API_BEGIN
    if (ctx->have_keys) drop_keys(ctx);
    keygen(ctx, seed);
    make_key(ctx, 0);
    make_key(ctx, 2 * ctx->N - 1);
    for (int i = 0; i < n_rot; i++) make_key(ctx, galois_for_rot(ctx, rot_steps[i]));
    if (ctx->bootstrap) {
        for (int inv = 0; inv < 2; inv++) {
            int nl = inv ? ctx->cts_levels : ctx->stc_levels;
            for (const LtDesc &lv : lt_levels(ctx, nl, inv))
                for (int r : lt_rotation_steps(ctx, lv)) make_key(ctx, galois_for_rot(ctx, r));
        }
    }
    CK(cudaStreamSynchronize(ctx->st));
    API_END
}

int he_keygen_softmax(he_ctx *ctx, int n, int m) {
    if (!ctx || n < 1 || m < 1 || (n & (n - 1)) || n % m || ctx->n0 % n) return HE_EINVAL;
    API_BEGIN
    REQUIRE(ctx->have_keys, HE_ENOKEY, "keygen first");
    int stride = (int)((long)m * ctx->n0 / n);
    for (int i = 0; (1 << i) < n / m; i++) make_key(ctx, galois_for_rot(ctx, (long)stride << i));
    CK(cudaStreamSynchronize(ctx->st));
    API_END
}

int he_encrypt(he_ctx *ctx, const double *x, size_t count, int n, int m, double M, uint64_t seed, he_ct *out) {
    if (!ctx || !x || !out || !out->data || n < 1 || m < 1 || (n & (n - 1)) || n % m || ctx->n0 % n || !(M > 0))
        return HE_EINVAL;
    size_t L = (size_t)m * ctx->n0 / n;
    if (count != L * (size_t)n) {
        ctx->err = "count must be L n with L = m N0 / n";
        return HE_EINVAL;
    }
    for (size_t i = 0; i < count; i++)
        if (!(x[i] <= 0.0 && x[i] >= -M)) {
            ctx->err = "inputs must lie in [-M, 0] (Assumption 3.5)";
            return HE_EINVAL;
        }
    API_BEGIN
    int top = ctx->user_top, per = n / m;
    double scale = (2.0 / M) * (double)ctx->mods[top];
    long cs = 2L * (top + 1) * ctx->N;
    for (int c = 0; c < m; c++) {
        std::vector<double2> z(ctx->n0, make_double2(0.0, 0.0));
        for (int t = 0; t < per; t++)
            for (size_t l = 0; l < L; l++) z[t * L + l].x = x[l * n + (size_t)c * per + t];
        encrypt_into(ctx, z, top, scale, seed, c, out->data + c * cs);
    }
    out->level = top;
    out->scale = scale;
    out->n_ct = m;
    CK(cudaStreamSynchronize(ctx->st));
    API_END
}

int he_decrypt(he_ctx *ctx, const he_ct *cts, int n, double *y, size_t count) {
    if (!ctx || !cts || !y || n < 1 || cts->n_ct < 1 || n % cts->n_ct || ctx->n0 % n) return HE_EINVAL;
    int m = cts->n_ct, per = n / m;
    size_t L = (size_t)m * ctx->n0 / n;
    if (count != L * (size_t)n) return HE_EINVAL;
    API_BEGIN
    DCt x = ct_view(ctx, cts);
    for (int c = 0; c < m; c++) {
        std::vector<double2> z = decrypt_slots(ctx, x, c);
        for (int t = 0; t < per; t++)
            for (size_t l = 0; l < L; l++) y[l * n + (size_t)c * per + t] = z[t * L + l].x;
    }
    API_END
}

int he_decrypt_slots(he_ctx *ctx, const he_ct *cts, int ct, double *slots) {
    if (!ctx || !cts || !slots || ct < 0 || ct >= cts->n_ct) return HE_EINVAL;
    API_BEGIN
    std::vector<double2> z = decrypt_slots(ctx, ct_view(ctx, cts), ct);
    memcpy(slots, z.data(), sizeof(double2) * ctx->n0);
    API_END
}

int he_encrypt_slots(he_ctx *ctx, const double *slots, int level, double scale, uint64_t seed, int ct_index, he_ct *out,
                     int ct) {
    if (!ctx || !slots || !out || !out->data || level < 0 || level >= ctx->nq || ct < 0 || ct >= out->n_ct)
        return HE_EINVAL;
    API_BEGIN
    std::vector<double2> z(ctx->n0);
    memcpy(z.data(), slots, sizeof(double2) * ctx->n0);
    encrypt_into(ctx, z, level, scale, seed, ct_index, out->data + (long)ct * 2 * (level + 1) * ctx->N);
    out->level = level;
    out->scale = scale;
    CK(cudaStreamSynchronize(ctx->st));
    API_END
}

static Plan plan_of(he_ctx *c, const he_softmax_plan *hp) {
    Plan p;
    p.n = hp->n;
    p.k = hp->k;
    p.M = hp->M;
    p.boost = hp->bts_boost > 0 ? hp->bts_boost : 1.0;
    p.exp_deg = hp->exp_deg;
    p.method = hp->method;
    p.exp_c.assign(hp->exp_coeffs, hp->exp_coeffs + hp->exp_deg + 1);
    const double *cp = hp->inv_coeffs;
    for (int j = 0; j < p.k; j++) {
        p.inv_deg.push_back(hp->inv_deg[j]);
        p.inv_c.emplace_back(cp, cp + hp->inv_deg[j] + 1);
        cp += hp->inv_deg[j] + 1;
        p.a.push_back(hp->inv_a[j]);
        p.b.push_back(hp->inv_b[j]);
        p.gs.push_back(hp->gain_s[j]);
        if (p.method == HE_SOFTMAX_ALG4) {
            p.expo.push_back(hp->exponent[j]);
            p.lam_max.push_back(hp->lam_max[j]);
            p.b_max.push_back(hp->b_max[j]);
        } else {
            p.gl.push_back(hp->gain_l[j]);
        }
    }
    (void)c;
    return p;
}

static int softmax_check(he_ctx *ctx, const he_softmax_plan *plan, const he_ct *cts, int groups = 1) {
    if (!ctx || !plan || !cts || !cts->data || cts->n_ct < 1 || plan->k < 1 || plan->k > 16) return HE_EINVAL;
    if (groups < 1 || cts->n_ct % groups) {
        ctx->err = "groups must divide the ciphertext count";
        return HE_EINVAL;
    }
    int m = cts->n_ct / groups, n = plan->n;
    if (n < 1 || (n & (n - 1)) || n % m || ctx->n0 % n) {
        ctx->err = "n must be a power of two dividing N/2, and m must divide n";
        return HE_EINVAL;
    }
    if (plan->method != HE_SOFTMAX_ALG2 && plan->method != HE_SOFTMAX_ALG4) {
        ctx->err = "plan method must be HE_SOFTMAX_ALG2 or HE_SOFTMAX_ALG4";
        return HE_EINVAL;
    }
    if (!plan->exp_coeffs || !plan->inv_deg || !plan->inv_coeffs || !plan->inv_a || !plan->inv_b ||
        !plan->gain_s || (plan->method == HE_SOFTMAX_ALG2 && !plan->gain_l) ||
        (plan->method == HE_SOFTMAX_ALG4 && (!plan->exponent || !plan->lam_max || !plan->b_max))) {
        ctx->err = "plan: a coefficient or gain array is missing";
        return HE_EINVAL;
    }
    if (plan->method == HE_SOFTMAX_ALG4 && !ctx->bootstrap) {
        ctx->err = "Alg. 4 needs a context with bootstrapping";
        return HE_EINVAL;
    }
    return HE_OK;
}

// the Softmax circuit on the ciphertexts of cts (groups independent groups), in place
static void softmax_inplace(he_ctx *ctx, const he_softmax_plan *plan, he_ct *cts, bool batched, int groups = 1) {
    int m = cts->n_ct / groups;
    Plan p = plan_of(ctx, plan);
    DCt in = ct_view(ctx, cts);
    std::vector<DCt> ys;
    if (batched) {
        ys.push_back(ct_copy(ctx, in));
    } else {
        REQUIRE(groups == 1, HE_EINVAL, "groups need the batched form");
        for (int i = 0; i < m; i++) ys.push_back(ct_copy(ctx, ct_sub(ctx, in, i)));
    }
    ys = p.method == HE_SOFTMAX_ALG4 ? softmax_run_b(ctx, p, ys, m, batched ? groups : 1)
                                     : softmax_run(ctx, p, ys, m, batched ? groups : 1);
    int lo = ys[0].level;
    long cs = 2L * (lo + 1) * ctx->N;
    if (batched) {
        CK(cudaMemcpyAsync(cts->data, ys[0].d, (size_t)cts->n_ct * cs * 8, cudaMemcpyDeviceToDevice, ctx->st));
    } else {
        for (int i = 0; i < m; i++)
            CK(cudaMemcpyAsync(cts->data + i * cs, ys[i].d, (size_t)cs * 8, cudaMemcpyDeviceToDevice, ctx->st));
    }
    cts->level = lo;
    cts->scale = ys[0].scale;
}

int he_softmax(he_ctx *ctx, const he_softmax_plan *plan, he_ct *cts, int batched) {
    int rc = softmax_check(ctx, plan, cts);
    if (rc) return rc;
    API_BEGIN
    softmax_inplace(ctx, plan, cts, batched != 0);
    API_END
}

int he_softmax_register(he_ctx *ctx, const he_softmax_plan *plan) {
    if (!ctx || !plan || plan->k < 1 || plan->k > 16 || plan->exp_deg < 0 || !plan->exp_coeffs || !plan->inv_deg ||
        !plan->inv_coeffs || !plan->inv_a || !plan->inv_b || !plan->gain_s)
        return HE_EINVAL;
    const bool b4 = plan->method == HE_SOFTMAX_ALG4;
    if (plan->method != HE_SOFTMAX_ALG2 && !b4) return HE_EINVAL;
    if (b4 ? (!plan->exponent || !plan->lam_max || !plan->b_max) : !plan->gain_l) return HE_EINVAL;
    const int k = plan->k;
    size_t nc = 0;
    for (int j = 0; j < k; j++) {
        if (plan->inv_deg[j] < 0) return HE_EINVAL;
        nc += plan->inv_deg[j] + 1;
    }
    he_ctx::PlanCopy &e = ctx->plans[std::make_tuple(plan->n, plan->M, plan->method)];
    e = he_ctx::PlanCopy{};
    e.exp_c.assign(plan->exp_coeffs, plan->exp_coeffs + plan->exp_deg + 1);
    e.inv_c.assign(plan->inv_coeffs, plan->inv_coeffs + nc);
    e.deg.assign(plan->inv_deg, plan->inv_deg + k);
    e.a.assign(plan->inv_a, plan->inv_a + k);
    e.b.assign(plan->inv_b, plan->inv_b + k);
    e.gs.assign(plan->gain_s, plan->gain_s + k);
    if (plan->gain_l) e.gl.assign(plan->gain_l, plan->gain_l + k);
    if (b4) {
        e.expo.assign(plan->exponent, plan->exponent + k);
        e.lam_max.assign(plan->lam_max, plan->lam_max + k);
        e.b_max.assign(plan->b_max, plan->b_max + k);
    }
    e.p = *plan;
    e.p.exp_coeffs = e.exp_c.data();
    e.p.inv_coeffs = e.inv_c.data();
    e.p.inv_deg = e.deg.data();
    e.p.inv_a = e.a.data();
    e.p.inv_b = e.b.data();
    e.p.gain_s = e.gs.data();
    e.p.gain_l = e.gl.empty() ? nullptr : e.gl.data();
    e.p.exponent = b4 ? e.expo.data() : nullptr;
    e.p.lam_max = b4 ? e.lam_max.data() : nullptr;
    e.p.b_max = b4 ? e.b_max.data() : nullptr;
    return HE_OK;
}

int he_softmax_nm(he_ctx *ctx, he_ct *cts, int n, double M, int method, int graph) {
    if (!ctx) return HE_EINVAL;
    auto it = ctx->plans.find(std::make_tuple(n, M, method));
    if (it == ctx->plans.end()) {
        ctx->err = "he_softmax_nm: no registered plan for this (n, M, method)";
        return HE_EINVAL;
    }
    return graph ? he_softmax_graph(ctx, &it->second.p, cts) : he_softmax(ctx, &it->second.p, cts, 1);
}

int he_softmax_grouped(he_ctx *ctx, const he_softmax_plan *plan, he_ct *cts, int groups) {
    int rc = softmax_check(ctx, plan, cts, groups);
    if (rc) return rc;
    API_BEGIN
    softmax_inplace(ctx, plan, cts, true, groups);
    API_END
}

// FNV-1a over the bytes of the plan's numbers: graphs are reused only for the same circuit
static uint64_t plan_hash(const he_softmax_plan *hp) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&h](const void *p, size_t n) {
        const unsigned char *b = (const unsigned char *)p;
        for (size_t i = 0; i < n; i++) h = (h ^ b[i]) * 1099511628211ull;
    };
    mix(&hp->n, sizeof hp->n);
    mix(&hp->k, sizeof hp->k);
    mix(&hp->M, sizeof hp->M);
    mix(&hp->bts_boost, sizeof hp->bts_boost);
    mix(&hp->exp_deg, sizeof hp->exp_deg);
    mix(hp->exp_coeffs, sizeof(double) * (hp->exp_deg + 1));
    mix(hp->inv_deg, sizeof(int) * hp->k);
    size_t nc = 0;
    for (int j = 0; j < hp->k; j++) nc += hp->inv_deg[j] + 1;
    mix(hp->inv_coeffs, sizeof(double) * nc);
    mix(hp->inv_a, sizeof(double) * hp->k);
    mix(hp->inv_b, sizeof(double) * hp->k);
    mix(hp->gain_s, sizeof(double) * hp->k);
    mix(&hp->method, sizeof hp->method);
    if (hp->method == HE_SOFTMAX_ALG4) {
        mix(hp->exponent, sizeof(double) * hp->k);
        mix(hp->lam_max, sizeof(double) * hp->k);
        mix(hp->b_max, sizeof(double) * hp->k);
    } else {
        mix(hp->gain_l, sizeof(double) * hp->k);
    }
    return h;
}

int he_softmax_graph(he_ctx *ctx, const he_softmax_plan *plan, he_ct *cts) {
    int rc = softmax_check(ctx, plan, cts);
    if (rc) return rc;
    API_BEGIN
    char key[160];
    snprintf(key, sizeof key, "%p:%d:%a:%d:%016llx", (void *)cts->data, cts->level, cts->scale, cts->n_ct,
             (unsigned long long)plan_hash(plan));
    auto it = ctx->graphs.find(key);
    if (it == ctx->graphs.end()) {
        // 1. an eager run on a copy fills the key, diagonal and mask caches (nothing is
        //    encoded or allocated outside the stream during the capture)
        {
            size_t words = (size_t)cts->n_ct * 2 * (cts->level + 1) * ctx->N;
            DPtr tmp = dalloc(ctx, words);
            CK(cudaMemcpyAsync(tmp.get(), cts->data, words * 8, cudaMemcpyDeviceToDevice, ctx->st));
            he_ct t = *cts;
            t.data = tmp.get();
            softmax_inplace(ctx, plan, &t, true);
        }
        // 2. capture the circuit on the context stream (temporaries become graph allocations)
        he_ctx::SmGraph gr;
        long l0 = ctx->launches, c0[5];
        for (int i = 0; i < 5; i++) c0[i] = ctx->cnt[i];
        he_ct out = *cts;
        cudaGraph_t graph = nullptr;
        if (!ctx->gstream) {
            CK(cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&ctx->gev_in, cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&ctx->gev_out, cudaEventDisableTiming));
        }
        cudaStream_t user = ctx->st;
        ctx->st = ctx->gstream;   // everything below is recorded into the graph
        // plain kernel edges in the graph: its replay hides launch latency by itself
        struct PdlOff {
            int prev = he_pdl_launch;
            PdlOff() { he_pdl_launch = 0; }
            ~PdlOff() { he_pdl_launch = prev; }
        } pdl_off;
        CK(cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal));
        ctx->capturing = true;
        ctx->cap_prof.clear();
        try {
            softmax_inplace(ctx, plan, &out, true);
        } catch (...) {
            ctx->capturing = false;
            cudaStreamEndCapture(ctx->st, &graph);
            ctx->st = user;
            if (graph) cudaGraphDestroy(graph);
            for (auto &r : ctx->cap_prof) {
                cudaEventDestroy(r.a);
                cudaEventDestroy(r.b);
            }
            ctx->cap_prof.clear();
            throw;
        }
        ctx->capturing = false;
        gr.prof.swap(ctx->cap_prof);
        cudaError_t ec = cudaStreamEndCapture(ctx->st, &graph);
        ctx->st = user;
        CK(ec);
        cudaError_t e = cudaGraphInstantiate(&gr.exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(e);
        gr.level = out.level;
        gr.scale = out.scale;
        gr.launches = ctx->launches - l0;
        for (int i = 0; i < 5; i++) gr.cnt[i] = ctx->cnt[i] - c0[i];
        // the capture only recorded the work: count it at each launch below
        ctx->launches = l0;
        for (int i = 0; i < 5; i++) ctx->cnt[i] = c0[i];
        it = ctx->graphs.emplace(key, gr).first;
    }
    he_ctx::SmGraph &gr = it->second;
    CK(cudaEventRecord(ctx->gev_in, ctx->st));
    CK(cudaStreamWaitEvent(ctx->gstream, ctx->gev_in, 0));
    CK(cudaGraphLaunch(gr.exec, ctx->gstream));
    CK(cudaEventRecord(ctx->gev_out, ctx->gstream));
    CK(cudaStreamWaitEvent(ctx->st, ctx->gev_out, 0));
    gr.replayed = true;
    ctx->launches += gr.launches;
    for (int i = 0; i < 5; i++) ctx->cnt[i] += gr.cnt[i];
    cts->level = gr.level;
    cts->scale = gr.scale;
    API_END
}

// ---- Alg. 4 split over shares of the main-thread ciphertexts (one share per device)
static int share_plan_check(he_ctx *ctx, const he_softmax_plan *plan, int m_total) {
    if (!ctx || !plan || plan->k < 1 || plan->k > 16 || plan->method != HE_SOFTMAX_ALG4 || !plan->exp_coeffs ||
        !plan->inv_deg || !plan->inv_coeffs || !plan->inv_a || !plan->inv_b || !plan->gain_s || !plan->exponent ||
        !plan->lam_max || !plan->b_max)
        return HE_EINVAL;
    int n = plan->n;
    if (m_total < 1 || n < 1 || (n & (n - 1)) || n % m_total || ctx->n0 % n || !ctx->bootstrap) {
        ctx->err = "split Softmax: Alg. 4 plan, a bootstrapping context, n a power of two dividing N/2 and m | n";
        return HE_EINVAL;
    }
    return HE_OK;
}

static void put_compact(he_ctx *ctx, const DCt &y, he_ct *out) {
    CK(cudaMemcpyAsync(out->data, y.d, (size_t)y.nct * y.cs(ctx) * 8, cudaMemcpyDeviceToDevice, ctx->st));
    out->level = y.level;
    out->scale = y.scale;
    out->n_ct = y.nct;
}

int he_softmax_share_exp(he_ctx *ctx, const he_softmax_plan *plan, he_ct *share) {
    int rc = share_plan_check(ctx, plan, 1);
    if (rc) return rc;
    if (!share || !share->data) return HE_EINVAL;
    API_BEGIN
    Plan p = plan_of(ctx, plan);
    std::vector<DCt> ys{ct_copy(ctx, ct_view(ctx, share))};
    alg4_exp(ctx, p, ys);
    put_compact(ctx, ys[0], share);
    API_END
}

int he_softmax_share_square_sum(he_ctx *ctx, const he_ct *ys, uint64_t *d) {
    if (!ctx || !ys || !d) return HE_EINVAL;
    API_BEGIN
    DCt y = ct_view(ctx, ys);
    DPtr t = tensor_sum(ctx, std::vector<DCt>{y}, y.nct, 1);
    CK(cudaMemcpyAsync(d, t.get(), (size_t)3 * (y.level + 1) * ctx->N * 8, cudaMemcpyDeviceToDevice, ctx->st));
    API_END
}

int he_softmax_aux_round(he_ctx *ctx, const he_softmax_plan *plan, int j, int m_total, const uint64_t *d_sum,
                         int level, double y_scale, int y0_level, double y0_scale, he_ct *lam, he_ct *lr) {
    int rc = share_plan_check(ctx, plan, m_total);
    if (rc) return rc;
    if (!d_sum || !lam || !lam->data || !lr || !lr->data || j < 1 || j > plan->k || level < 1 || level >= ctx->nq ||
        y0_level < 1 || y0_level >= ctx->nq)
        return HE_EINVAL;
    API_BEGIN
    Plan p = plan_of(ctx, plan);
    int L = level + 1;
    DPtr dr = dalloc(ctx, (size_t)3 * L * ctx->N);
    {
        ProfScope ps_(ctx, "elementwise", 0);
        klaunch(k_reduce_limbs, grid_for(ctx, (long)3 * L << ctx->logN), 256, 0, ctx->st)(dr.get(), d_sum, 3 * L, L, qmap(L),
                                                                                   ctx->d_mods, ctx->logN);
    }
    he_ctx *c = ctx;
    LAUNCH_CHECK();
    DCt S = relin_sum(ctx, dr.get(), level, 1, y_scale);
    DCt lam_c;
    bool have_lam = j > 1;
    if (have_lam) lam_c = ct_view(ctx, lam);
    DCt out = alg4_aux(ctx, p, j, S, m_total, y0_level, y0_scale, lam_c, have_lam);
    put_compact(ctx, lam_c, lam);
    put_compact(ctx, out, lr);
    API_END
}

int he_softmax_share_update(he_ctx *ctx, const he_softmax_plan *plan, int j, const he_ct *lr, const he_ct *y0,
                            he_ct *ys) {
    int rc = share_plan_check(ctx, plan, 1);
    if (rc) return rc;
    if (!lr || !y0 || !ys || !ys->data || j < 1 || j > plan->k) return HE_EINVAL;
    API_BEGIN
    DCt l = ct_view(ctx, lr), y = ct_view(ctx, y0);
    REQUIRE(l.nct == 1, HE_EINVAL, "lr must be one ciphertext");
    REQUIRE(ys->data != y0->data, HE_EINVAL, "ys must not be y0's buffer");
    std::vector<DCt> out{y}, in{y};
    alg4_update(ctx, j, l, in, out, y.nct, 1);
    put_compact(ctx, out[0], ys);
    API_END
}

int he_ntt(he_ctx *ctx, uint64_t *data, int n_poly, int n_limb, int inverse) {
    if (!ctx || !data || n_poly < 1 || n_limb < 1 || n_limb > ctx->nq) return HE_EINVAL;
    API_BEGIN
    ntt(ctx, data, n_poly * n_limb, qmap(n_limb), (long)n_limb * ctx->N, inverse != 0);
    API_END
}

int he_ct_to_coeff(he_ctx *ctx, const he_ct *x, uint64_t *host) {
    if (!ctx || !x || !x->data || !host || x->level < 0 || x->level >= ctx->nq) return HE_EINVAL;
    API_BEGIN
    int L = x->level + 1;
    size_t words = (size_t)x->n_ct * 2 * L * ctx->N;
    DPtr t = dalloc(ctx, words);
    CK(cudaMemcpyAsync(t.get(), x->data, words * 8, cudaMemcpyDeviceToDevice, ctx->st));
    ntt(ctx, t.get(), x->n_ct * 2 * L, qmap(L), (long)L * ctx->N, true);
    CK(cudaMemcpyAsync(host, t.get(), words * 8, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    API_END
}

int he_ct_from_coeff(he_ctx *ctx, const uint64_t *host, he_ct *x) {
    if (!ctx || !x || !x->data || !host || x->level < 0 || x->level >= ctx->nq || x->n_ct < 1) return HE_EINVAL;
    API_BEGIN
    int L = x->level + 1;
    size_t words = (size_t)x->n_ct * 2 * L * ctx->N;
    CK(cudaMemcpyAsync(x->data, host, words * 8, cudaMemcpyHostToDevice, ctx->st));
    ntt(ctx, x->data, x->n_ct * 2 * L, qmap(L), (long)L * ctx->N, false);
    CK(cudaStreamSynchronize(ctx->st));
    API_END
}

int he_encode(he_ctx *ctx, const double *slots, double scale, int level, uint64_t *pt) {
    if (!ctx || !slots || !pt || level < 0 || level >= ctx->nq) return HE_EINVAL;
    API_BEGIN
    std::vector<double2> z(ctx->n0);
    memcpy(z.data(), slots, sizeof(double2) * ctx->n0);
    DPtr d = encode(ctx, z, scale, level);
    CK(cudaMemcpyAsync(pt, d.get(), (size_t)(level + 1) * ctx->N * 8, cudaMemcpyDeviceToDevice, ctx->st));
    API_END
}

int he_add(he_ctx *ctx, he_ct *a, const he_ct *b) {
    if (!ctx || !a || !b) return HE_EINVAL;
    API_BEGIN
    DCt x = ct_view(ctx, a);
    ct_add_inplace(ctx, x, ct_view(ctx, b));
    API_END
}

int he_mul_plain(he_ctx *ctx, he_ct *a, const uint64_t *pt) {
    if (!ctx || !a || !pt) return HE_EINVAL;
    API_BEGIN
    DCt x = ct_view(ctx, a);
    ct_mul_plain(ctx, x, pt);
    API_END
}

static void put_out(he_ctx *ctx, const DCt &y, he_ct *out) {
    REQUIRE(out->data, HE_EINVAL, "output buffer");
    CK(cudaMemcpyAsync(out->data, y.d, (size_t)y.nct * y.cs(ctx) * 8, cudaMemcpyDeviceToDevice, ctx->st));
    out->level = y.level;
    out->scale = y.scale;
    out->n_ct = y.nct;
}

int he_rescale(he_ctx *ctx, const he_ct *a, he_ct *out) {
    if (!ctx || !a || !out) return HE_EINVAL;
    API_BEGIN
    put_out(ctx, rescale(ctx, ct_view(ctx, a)), out);
    API_END
}

int he_rescale_noalloc(he_ctx *ctx, const he_ct *a, he_ct *out) {
    if (!ctx || !a || !out || !a->data || !out->data || a->n_ct < 1) return HE_EINVAL;
    if (a->level < 0 || a->level >= ctx->nq) {
        ctx->err = "he_rescale_noalloc: level must be in [0, n_q)";
        return HE_EINVAL;
    }
    if (a->level == 0) {
        ctx->err = "he_rescale_noalloc: rescale at level 0";
        return HE_ELEVEL;
    }
    size_t need = (size_t)2 * a->n_ct * (a->level + 1) * ctx->N;
    {
        // the final pass reads a with stride level+1 limbs and writes out with stride level:
        // any overlap of the two byte ranges would let it overwrite limbs not yet read
        uintptr_t a0 = (uintptr_t)a->data, a1 = a0 + need * 8;
        uintptr_t o0 = (uintptr_t)out->data, o1 = o0 + (size_t)2 * a->n_ct * a->level * ctx->N * 8;
        if (o0 < a1 && a0 < o1) {
            ctx->err = "he_rescale_noalloc: output must not overlap the input";
            return HE_EINVAL;
        }
    }
    if (need > HE_NOALLOC_SCRATCH_WORDS) {
        char b[160];
        snprintf(b, sizeof b, "he_rescale_noalloc: needs %zu scratch words, the fixed scratch holds %u "
                 "(2 n_ct (level+1) N <= %u)", need, HE_NOALLOC_SCRATCH_WORDS, HE_NOALLOC_SCRATCH_WORDS);
        ctx->err = b;
        return HE_EINVAL;
    }
    API_BEGIN
    rescale_noalloc(ctx, ct_view(ctx, a), out->data);
    out->level = a->level - 1;
    out->scale = a->scale / (double)ctx->mods[a->level];
    out->n_ct = a->n_ct;
    API_END
}

int he_hmult(he_ctx *ctx, const he_ct *a, const he_ct *b, he_ct *out) {
    if (!ctx || !a || !b || !out) return HE_EINVAL;
    API_BEGIN
    put_out(ctx, hmult(ctx, ct_view(ctx, a), ct_view(ctx, b)), out);
    API_END
}

int he_relinearize(he_ctx *ctx, const uint64_t *d, int level, int n_ct, he_ct *out) {
    if (!ctx || !d || !out || level < 0 || level >= ctx->nq || n_ct < 1) return HE_EINVAL;
    API_BEGIN
    put_out(ctx, relinearize(ctx, d, level, n_ct, 1.0), out);
    API_END
}

int he_rotate(he_ctx *ctx, const he_ct *a, int r, he_ct *out) {
    if (!ctx || !a || !out) return HE_EINVAL;
    API_BEGIN
    put_out(ctx, rotate(ctx, ct_view(ctx, a), galois_for_rot(ctx, r)), out);
    API_END
}

int he_conjugate(he_ctx *ctx, const he_ct *a, he_ct *out) {
    if (!ctx || !a || !out) return HE_EINVAL;
    API_BEGIN
    put_out(ctx, rotate(ctx, ct_view(ctx, a), 2 * ctx->N - 1), out);
    API_END
}

int he_poly_eval(he_ctx *ctx, const he_ct *u, const double *coeffs, int deg, int level_out, double scale_out, he_ct *out) {
    if (!ctx || !u || !coeffs || !out || deg < 1 || level_out < 0) return HE_EINVAL;
    API_BEGIN
    std::vector<double> cf(coeffs, coeffs + deg + 1);
    put_out(ctx, poly_eval(ctx, ct_view(ctx, u), cf, level_out, scale_out), out);
    API_END
}

int he_lintrans(he_ctx *ctx, const he_ct *a, int nlev, int inverse, int which, double gain, double pt_scale, he_ct *out) {
    if (!ctx || !a || !out || nlev < 1 || which < 0 || which >= nlev) return HE_EINVAL;
    API_BEGIN
    std::vector<LtDesc> lv = lt_levels(ctx, nlev, inverse);
    put_out(ctx, lt_eval_level(ctx, ct_view(ctx, a), lv[which], gain, pt_scale), out);
    API_END
}

int he_bootstrap(he_ctx *ctx, const he_ct *a, double gain, double out_scale, he_ct *out) {
    if (!ctx || !a || !out) return HE_EINVAL;
    API_BEGIN
    put_out(ctx, bootstrap(ctx, ct_view(ctx, a), gain, out_scale), out);
    API_END
}

int he_mod_raise(he_ctx *ctx, const he_ct *a, int top, he_ct *out) {
    if (!ctx || !a || !out || top < 0 || top >= ctx->nq) return HE_EINVAL;
    API_BEGIN
    put_out(ctx, mod_raise(ctx, ct_view(ctx, a), top), out);
    API_END
}

int he_autotune(he_ctx *ctx, const int *levels, int n_levels, const int *ncts, int n_ncts, int reps) {
    if (!ctx || !levels || !ncts || n_levels < 1 || n_ncts < 1 || reps < 1) return HE_EINVAL;
    for (int i = 0; i < n_levels; i++)
        if (levels[i] < 1 || levels[i] >= ctx->nq) return HE_EINVAL;
    for (int i = 0; i < n_ncts; i++)
        if (ncts[i] < 1 || ncts[i] > 4096) return HE_EINVAL;
    API_BEGIN
    autotune(ctx, std::vector<int>(levels, levels + n_levels), std::vector<int>(ncts, ncts + n_ncts), reps);
    API_END
}

int he_tune_table(const he_ctx *ctx, char *buf, size_t len) {
    if (!ctx || !buf || len == 0) return HE_EINVAL;
    std::string out;
    for (const auto &kv : ctx->tune) {
        char line[128];
        snprintf(line, sizeof line, "%d %d %d %d %.4f %.4f\n", std::get<0>(kv.first), std::get<1>(kv.first),
                 std::get<2>(kv.first), kv.second.choice, kv.second.ms[0], kv.second.ms[1]);
        out += line;
    }
    if (out.size() >= len) return HE_EINVAL;
    memcpy(buf, out.c_str(), out.size() + 1);
    return HE_OK;
}

int he_tune_force(he_ctx *ctx, int op, int choice) {
    if (!ctx || op < 0 || op > HE_TUNE_NTT_1PASS || choice < -1 || choice > 1) return HE_EINVAL;
    ctx->tune_force[op] = choice;
    return HE_OK;
}

int he_counters(const he_ctx *ctx, long *out5) {
    if (!ctx || !out5) return HE_EINVAL;
    for (int i = 0; i < 5; i++) out5[i] = ctx->cnt[i];
    return HE_OK;
}

long he_launch_count(const he_ctx *ctx) { return ctx ? ctx->launches : -1; }

int he_profile_kernel(he_ctx *ctx, const char *name) {
    if (!ctx) return HE_EINVAL;
    ctx->prof_name = name ? name : "";
    ctx->prof_used = 0;
    ctx->prof_bytes = 0;
    return HE_OK;
}

int he_profile_read(he_ctx *ctx, double *total_ms, long *launches, double *bytes) {
    if (!ctx || !total_ms || !launches || !bytes) return HE_EINVAL;
    API_BEGIN
    CK(cudaStreamSynchronize(ctx->st));
    double t = 0, by = ctx->prof_bytes;
    long n = (long)ctx->prof_used;
    for (size_t i = 0; i < ctx->prof_used; i++) {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, ctx->prof_ev[i].first, ctx->prof_ev[i].second));
        t += ms;
    }
    for (auto &kv : ctx->graphs) {
        if (!kv.second.replayed) continue;
        for (const auto &r : kv.second.prof) {
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, r.a, r.b));
            t += ms;
            by += r.bytes;
            n++;
        }
        kv.second.replayed = false;
    }
    *total_ms = t;
    *launches = n;
    *bytes = by;
    ctx->prof_used = 0;
    ctx->prof_bytes = 0;
    API_END
}

int he_profile_breakdown(he_ctx *ctx, char *buf, size_t len) {
    if (!ctx || !buf || len == 0) return HE_EINVAL;
    API_BEGIN
    CK(cudaStreamSynchronize(ctx->st));
    std::map<std::string, std::tuple<long, double, double>> fam;
    for (size_t i = 0; i < ctx->prof_used; i++) {
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, ctx->prof_ev[i].first, ctx->prof_ev[i].second));
        auto &f = fam[ctx->prof_fam[i]];
        std::get<0>(f)++;
        std::get<1>(f) += ms;
        std::get<2>(f) += ctx->prof_b[i];
        auto &ph = fam[std::string("phase:") + ctx->prof_ph[i]];
        std::get<0>(ph)++;
        std::get<1>(ph) += ms;
        auto &pf = fam[std::string("pf:") + ctx->prof_ph[i] + ":" + ctx->prof_fam[i]];
        std::get<0>(pf)++;
        std::get<1>(pf) += ms;
        std::get<2>(pf) += ctx->prof_b[i];
    }
    for (auto &kv : ctx->graphs) {
        if (!kv.second.replayed) continue;
        for (const auto &r : kv.second.prof) {
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, r.a, r.b));
            auto &f = fam[r.fam];
            std::get<0>(f)++;
            std::get<1>(f) += ms;
            std::get<2>(f) += r.bytes;
        }
        kv.second.replayed = false;
    }
    std::string out;
    for (const auto &kv : fam) {
        char line[160];
        snprintf(line, sizeof line, "%s %ld %.6f %.6e\n", kv.first.c_str(), std::get<0>(kv.second),
                 std::get<1>(kv.second), std::get<2>(kv.second));
        out += line;
    }
    ctx->prof_used = 0;
    ctx->prof_bytes = 0;
    REQUIRE(out.size() < len, HE_EINVAL, "he_profile_breakdown: buffer too small");
    memcpy(buf, out.c_str(), out.size() + 1);
    API_END
}

int he_selftest_bounded_wait(he_ctx *ctx, long max_iter) {
    if (!ctx || max_iter < 1) return HE_EINVAL;
    he_ctx *c = ctx;
    API_BEGIN
    DPtr b = dalloc(ctx, 1);
    int *flag = (int *)b.get(), *status = flag + 1;
    CK(cudaMemsetAsync(b.get(), 0, 8, ctx->st));
    klaunch(k_bounded_wait, 1, 32, 0, ctx->st)(flag, status, max_iter);
    LAUNCH_CHECK();
    int hs = 0;
    CK(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (hs == 2) {
        ctx->err = "bounded wait gave up";
        return HE_ETIMEOUT;
    }
    API_END
}

}  // extern "C"
