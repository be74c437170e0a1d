// C ABI of libgol: handles, host<->device transfers, planning of packed
// steps into units, the plan/graph cache and the autotune table.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_set>
#include <vector>

#include "gol_internal.h"

using namespace gol;

struct gol_board {
    int64_t rows = 0, cols = 0, words = 0;   // words per row (packed)
    int torus = 1;
    int layout = GOL_LAYOUT_PACKED;
    void *buf[2] = {nullptr, nullptr};
    int32_t *dev_cur = nullptr;              // device copy of `cur`
    int cur = 0;                             // host mirror
    int64_t generation = 0;
    size_t buf_bytes = 0;
    void *(*alloc_fn)(size_t, void *) = nullptr;
    void (*free_fn)(void *, void *) = nullptr;
    void *alloc_ctx = nullptr;
    uint64_t serial = 0;                     // identity for the plan cache
    uint64_t batch_stamp = 0;                // last batch call that listed the board (repeat check)
    // Packed boards may be stored transposed (stored row c holds column c of
    // the board): the step is symmetric under transposition, and a board
    // whose columns fit the warp lanes better that way runs faster.  The
    // stored geometry is srows x swords; the interchange layout is always the
    // board's own rows x words.
    int transposed = 0;
    int64_t srows = 0, swords = 0;
    // A packed board whose width is not a multiple of 64 (its height must
    // be) is always stored transposed, so that its stored rows are whole
    // words; it has no packed interchange layout (words = 0).
    int odd_width = 0;
    // A packed board with neither side a multiple of 64 keeps its rows as
    // ceil(cols / 64) words, the last word holding last_bits columns and zero
    // padding (see the masked variant of the step kernel).  Its packed
    // interchange layout has that many words per row as well.
    int masked = 0;
    int last_bits = 0;
    // byte boards: captured graphs of 64 generations, per starting buffer
    cudaGraphExec_t byte_graph[2] = {nullptr, nullptr};
    cudaStream_t byte_graph_stream = nullptr;
};

namespace {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
thread_local std::string t_err;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(GOL_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CU(expr)                                              \
    do {                                                      \
        cudaError_t e_ = (expr);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #expr);   \
    } while (0)

// ---------------------------------------------------------------------------
// process state
// ---------------------------------------------------------------------------
std::mutex g_mu;
cudaStream_t g_stream = nullptr;
void *(*g_alloc)(size_t, void *) = nullptr;
void (*g_free)(void *, void *) = nullptr;
void *g_alloc_ctx = nullptr;
int64_t g_opt_k = 0, g_opt_rows = 0, g_opt_graphs = 1, g_opt_timeout_ms = 5000, g_opt_orient = 0;
int64_t g_opt_chain = 0;     // chain cap, per mille of the average work per warp slot (0 = auto)
int64_t g_opt_variant = -1;  // step kernel variant (see launch_persistent), -1 = default
int64_t g_opt_zero_copy = 1; // many-board transfers read / write pinned host buffers in place
int64_t g_opt_byte_cluster = 1; // byte boards that fit one cluster's shared memory step there
int64_t g_opt_critical = -1;    // permille of the longest chain from which a queued pass is
                                // critical; -1: 750 for several boards, none for one board
uint64_t g_serial = 0;

struct DeviceState {
    bool ready = false;
    int device = -1;
    int sms = 0;
    int64_t l2 = 0;
    int clock_khz = 0;
    int32_t *sticky = nullptr;   // process-wide device error word
};
DeviceState g_dev;

int ensure_device() {
    if (g_dev.ready) return GOL_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice (no CUDA device?)");
    cudaDeviceProp p;
    CU(cudaGetDeviceProperties(&p, dev));
    g_dev.device = dev;
    g_dev.sms = p.multiProcessorCount;
    g_dev.l2 = p.l2CacheSize;
    int clk = 0;
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
    g_dev.clock_khz = clk;
    CU(cudaMalloc(&g_dev.sticky, sizeof(int32_t)));
    CU(cudaMemset(g_dev.sticky, 0, sizeof(int32_t)));
    g_dev.ready = true;
    return GOL_OK;
}

// allocation through the hook of the caller (board) or the process
void *dev_alloc(size_t n, void *(*af)(size_t, void *), void *ctx) {
    if (n == 0) n = 1;
    if (af) return af(n, ctx);
    void *p = nullptr;
    if (cudaMalloc(&p, n) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}
void dev_free(void *p, void (*ff)(void *, void *), void *ctx) {
    if (!p) return;
    if (ff)
        ff(p, ctx);
    else
        cudaFree(p);
}

void defer_free(void *p, void (*ff)(void *, void *), void *ctx);

// ---------------------------------------------------------------------------
// page-locked staging of table uploads
// ---------------------------------------------------------------------------
// A launch uploads tables built on the host (a unit plan, a transfer plan).
// A cudaMemcpyAsync from pageable memory may wait for the work already
// queued on the stream before it copies, which would hold the caller until
// the previous launch has finished; a copy from page-locked memory is only
// queued.  Staging blocks are kept for reuse (page-locked allocation is
// slow; they live as long as the process) and handed out again once an
// event recorded behind their last copy has completed.
struct StageBlock {
    char *p = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
    bool pending = false;
};
std::vector<StageBlock> &g_stage = *new std::vector<StageBlock>();
constexpr size_t kStageBlocks = 32;                  // a launch and a transfer plan per tick, a few ticks ahead
constexpr size_t kStageMin = size_t(256) << 10;

struct Upload {
    void *dst;           // device
    const void *src;     // host
    size_t n;            // bytes
};

// A free staging block of at least `total` bytes, or null (none free and no
// room for another).
StageBlock *stage_block(size_t total) {
    StageBlock *b = nullptr;
    for (auto &s : g_stage) {
        if (s.cap < total) continue;
        if (s.pending) {
            if (cudaEventQuery(s.ev) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            s.pending = false;
        }
        if (!b || s.cap < b->cap) b = &s;
    }
    if (b || g_stage.size() >= kStageBlocks) return b;
    StageBlock s;
    s.cap = kStageMin;
    while (s.cap < total) s.cap *= 2;
    if (cudaHostAlloc((void **)&s.p, s.cap, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeHost(s.p);
        return nullptr;
    }
    g_stage.push_back(s);
    return &g_stage.back();
}

// Queues the copies `parts` on the library's stream through one staging
// block (each part at a 16-byte offset).  While the stream is being
// captured, or when no block is free, the parts are copied from where they
// are.
cudaError_t upload(std::initializer_list<Upload> parts) {
    size_t total = 0;
    for (const Upload &u : parts) total += (u.n + 15) & ~size_t(15);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusActive;
    if (cudaStreamIsCapturing(g_stream, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;
    }
    StageBlock *b = (cs == cudaStreamCaptureStatusNone && total > 0) ? stage_block(total) : nullptr;
    size_t off = 0;
    for (const Upload &u : parts) {
        if (u.n == 0) continue;
        const void *src = u.src;
        if (b) {
            std::memcpy(b->p + off, u.src, u.n);
            src = b->p + off;
            off += (u.n + 15) & ~size_t(15);
        }
        cudaError_t e = cudaMemcpyAsync(u.dst, src, u.n, cudaMemcpyHostToDevice, g_stream);
        if (e != cudaSuccess) {
            if (b) cudaStreamSynchronize(g_stream);   // copies already queued from the block have run
            return e;
        }
    }
    if (b) {
        cudaError_t e = cudaEventRecord(b->ev, g_stream);
        if (e != cudaSuccess) {
            cudaStreamSynchronize(g_stream);
            return e;
        }
        b->pending = true;
    }
    return cudaSuccess;
}

// scoped temporary device buffer using the process allocator.  With an
// allocator hook the buffer is returned once the work queued on the stream
// so far has run (an event, see defer_free): the hook's allocator may hand
// it out again to work on another stream.
struct Scratch {
    void *p = nullptr;
    void *(*af)(size_t, void *) = g_alloc;
    void (*ff)(void *, void *) = g_free;
    void *ctx = g_alloc_ctx;
    explicit Scratch(size_t n) { p = dev_alloc(n, af, ctx); }
    ~Scratch() {
        if (p) {
            if (!ff) {
                cudaStreamSynchronize(g_stream);
                dev_free(p, ff, ctx);
            } else {
                defer_free(p, ff, ctx);
            }
        }
    }
};

// read and clear the sticky device error
int take_sticky() {
    if (!g_dev.ready) return GOL_OK;
    int32_t v = 0;
    cudaError_t e = cudaMemcpy(&v, g_dev.sticky, sizeof v, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading device status");
    if (v != 0) {
        int32_t z = 0;
        cudaMemcpy(g_dev.sticky, &z, sizeof z, cudaMemcpyHostToDevice);
        return fail(v, "a device-side bounded wait gave up (status %d); results are not valid", v);
    }
    return GOL_OK;
}

int sync_stream() {
    CU(cudaStreamSynchronize(g_stream));
    return take_sticky();
}

bool valid(gol_handle h) { return h != nullptr && h->rows > 0; }
uint64_t g_batch_stamp = 0;   // gol_step_batch calls so far (under g_mu)

// ---------------------------------------------------------------------------
// autotune table
// ---------------------------------------------------------------------------
struct TuneEntry {
    int k;
    int rows;
};
std::map<std::pair<int, int>, TuneEntry> g_tune;

int ilog2_ceil(int64_t x) {
    int l = 0;
    while ((int64_t(1) << l) < x) ++l;
    return l;
}
std::pair<int, int> size_class(int64_t rows, int64_t cols) {
    const int64_t w = (cols + 63) / 64;
    const int wc = w <= 32 ? (int)w : 32 + ilog2_ceil(w);
    return {ilog2_ceil(rows), wc};
}
TuneEntry tune_lookup(int64_t rows, int64_t cols) {
    auto it = g_tune.find(size_class(rows, cols));
    TuneEntry t{6, 128};
    if (it != g_tune.end()) t = it->second;
    if (g_opt_k) t.k = (int)g_opt_k;
    if (g_opt_rows) t.rows = (int)g_opt_rows;
    return t;
}

// ---------------------------------------------------------------------------
// planning
// ---------------------------------------------------------------------------
struct Plan {
    std::vector<gol_handle> hs;
    std::vector<int64_t> gens;
    std::vector<uint64_t> serials;
    int K = 8;
    bool torus = true;
    int64_t opt_k = 0, opt_rows = 0, opt_chain = 0, opt_variant = 0, opt_critical = 0;
    int variant = 0;
    // population trace: every board's generation count is a whole number of
    // sampling periods of `every` generations; pop_first[i] is board i's
    // first sample slot (0 = no trace)
    int64_t every = 0;
    std::vector<int32_t> pop_first;
    bool masked = false;   // the boards have a masked last word (one launch holds only such boards or none)
    // host copies
    std::vector<BoardDesc> boards;
    std::vector<UnitDesc> units;
    std::vector<int32_t> init_order; // units by the queue ring of their first pass
    std::vector<int32_t> npass;      // per board
    int64_t total_tasks = 0;
    // device memory
    void *dmem = nullptr;
    size_t dbytes = 0;
    PersistArgs args{};
    int grid = 1;
    cudaGraphExec_t graph = nullptr;
    cudaStream_t graph_stream = nullptr;
    bool no_graph = false;
    uint64_t uses = 0;
    void (*free_fn)(void *, void *) = nullptr;
    void *alloc_ctx = nullptr;
    ~Plan() {
        if (graph) cudaGraphExecDestroy(graph);
        if (dmem) dev_free(dmem, free_fn, alloc_ctx);
    }
};

// generations-per-pass values with a kernel instantiation (persist_k*.cu)
#define GOL_FOR_EACH_K(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(16)
constexpr int kKs[] = {1, 2, 3, 4, 5, 6, 7, 8, 16};

bool is_supported_k(int k) {
    for (int v : kKs)
        if (v == k) return true;
    return false;
}
int supported_k(int k) {
    int s = 1;
    for (int v : kKs)
        if (v <= k) s = v;
    return s;
}
// Kernel variant of a plan: the window rotation by renaming (1) measured
// faster than register moves (0) on both the 4096-board batch and a 16384^2
// board once the join-counter scheduler removed most per-pass overhead.
// At K = 8 a launch with at least 8 units per warp of the unrestricted
// kernel (two warps per scheduler) takes variant 3, held to three warps per
// scheduler: measured on a 131072^2 board (35k units) 45.2k against 39.8k
// GCUPS, while a 16384^2 board (2304 units) keeps 35.7k with variant 1
// against 32.5k with variant 3.
int plan_variant(int K, int64_t units_estimate) {
    if (g_opt_variant >= 0) return (int)g_opt_variant;
    if (K == 8 && units_estimate >= 8LL * g_dev.sms * 8) return 3;
    return 1;
}

cudaError_t occupancy_for(int K, bool torus, int v, int *bps) {
    switch (K) {
#define X(KV) \
    case KV: return persistent_occupancy<KV>(torus, v, bps);
        GOL_FOR_EACH_K(X)
#undef X
    }
    return cudaErrorInvalidValue;
}
cudaError_t launch_for(int K, const PersistArgs &a, bool torus, int variant, int grid, cudaStream_t s) {
    switch (K) {
#define X(KV) \
    case KV: return launch_persistent<KV>(a, torus, variant, grid, s);
        GOL_FOR_EACH_K(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

// Units of one board: nb balanced row blocks (block i = [R*i/nb, R*(i+1)/nb))
// times nt word tiles.
struct UnitGrid {
    int nb, nt, S;
    bool full;
};

UnitGrid unit_grid(int64_t rows, int64_t words, int K, int tile_rows) {
    UnitGrid g;
    const int R = (int)rows, W = (int)words;
    g.full = W <= 32;
    g.S = g.full ? std::max(1, 32 / W) : 1;
    g.nt = g.full ? 1 : (W + kTileWords - 1) / kTileWords;
    // rows per unit: S segments of tile_rows rows (full rows) or tile_rows (tiles)
    const int64_t target = (int64_t)g.S * std::max(1, tile_rows);
    g.nb = (int)std::max<int64_t>(1, (R + target - 1) / target);
    // with more than one block every block must be >= K rows so that a halo
    // reaches only the adjacent blocks
    if (g.nb > 1 && R / g.nb < K) g.nb = std::max(1, R / K);
    return g;
}

// Writes the g.nb * g.nt units of a board to out[0..); unit ids are
// first + index.  `seam` > 0 rotates the word tiles by that many words
// (tile 0 starts at word W - seam and wraps), so that on a torus whose
// last word is partial that word and word 0 are output words of one tile
// rather than another tile's halo words.  Uses no dynamic memory.
void fill_units(int64_t rows, int64_t words, int bindex, const UnitGrid &g, UnitDesc *out, int first, int seam = 0) {
    const int R = (int)rows, W = (int)words, nb = g.nb, nt = g.nt, S = g.S;
    for (int i = 0; i < nb; ++i) {
        const int r0 = (int)((int64_t)R * i / nb), r1 = (int)((int64_t)R * (i + 1) / nb);
        const int bh = r1 - r0;
        for (int t = 0; t < nt; ++t) {
            UnitDesc u{};
            u.board = bindex;
            u.r0 = r0;
            u.r_end = r1;
            if (g.full) {
                u.mode = kUnitFull;
                u.H = (bh + S - 1) / S;
                u.S = (bh + u.H - 1) / u.H;
                u.w0 = 0;
                u.U = W;
            } else {
                u.mode = kUnitTiled;
                u.H = bh;
                u.S = 1;
                const int lo = (int)((int64_t)W * t / nt);
                u.U = (int)((int64_t)W * (t + 1) / nt) - lo;
                u.w0 = (lo + W - seam) % W;
            }
            // neighbours: adjacent row blocks x adjacent tiles (wrapping), minus self
            u.nnb = 0;
            for (int a = -1; a <= 1; ++a)
                for (int b = -1; b <= 1; ++b) {
                    const int ii = ((i + a) % nb + nb) % nb, tt = ((t + b) % nt + nt) % nt;
                    const int id = first + ii * nt + tt;
                    if (id == first + i * nt + t) continue;
                    bool seen = false;
                    for (int k = 0; k < u.nnb; ++k) seen = seen || u.nb[k] == id;
                    if (!seen) u.nb[u.nnb++] = id;
                }
            out[i * nt + t] = u;
        }
    }
}

// A board's pass length for the queue: its tallest unit's rows per pass,
// H + 2K (the same for all units of the board, so a claimer classifies a
// neighbour's pass from its own record).
void set_board_cost(UnitDesc *us, int n, int K) {
    int h = 0;
    for (int i = 0; i < n; ++i) h = std::max(h, us[i].H);
    for (int i = 0; i < n; ++i) us[i].cost = h + 2 * K;
}

// Queue layout of a launch (see PersistArgs): a pass is critical when the
// rest of its unit's chain, (npass - pass + 1) * cost, is at least hi_thr =
// GOL_OPT_CRITICAL_PERMILLE of the longest chain (0: no critical passes).
// Counts the critical passes (the critical ring's size) and lists the units
// by the ring of their first pass, critical first, each in unit (LPT) order,
// into init_out[0 .. nunits).  Units of a board are consecutive; npass_of(b)
// is board b's pass count.  Uses no dynamic memory.
// Measured on the 4096-board batch: 750 permille 34.9k GCUPS, 500 34.7k,
// 350 34.2k, 250 34.0k, none 33.7k; on one board (equal chains) it changes
// nothing and is off.
template <typename NpassOf>
void plan_rings(const UnitDesc *units, int nunits, size_t nboards, NpassOf npass_of, PersistArgs &a,
                int32_t *init_out) {
    int64_t maxchain = 1;
    for (int u = 0; u < nunits; ++u)
        maxchain = std::max(maxchain, (int64_t)npass_of(units[u].board) * units[u].cost);
    const int64_t permille = g_opt_critical >= 0 ? g_opt_critical : (nboards > 1 ? 750 : 0);
    a.hi_thr = permille > 0 ? std::max<int64_t>(1, (maxchain * permille + 999) / 1000) : INT64_MAX;
    int64_t hi_cap = 0;
    int32_t hi_init = 0;
    for (int u = 0; u < nunits; ++u) {
        const int64_t np = npass_of(units[u].board), cost = std::max(1, units[u].cost);
        const int64_t need = a.hi_thr == INT64_MAX ? np + 1 : (a.hi_thr + cost - 1) / cost;   // rest >= need passes
        hi_cap += std::max<int64_t>(0, std::min<int64_t>(np, np + 1 - need));
        if (np * cost >= a.hi_thr) ++hi_init;
    }
    a.hi_cap = (int32_t)hi_cap;
    a.hi_init = hi_init;
    int k = 0;
    for (int pass = 0; pass < 2; ++pass)
        for (int u = 0; u < nunits; ++u) {
            const bool hi = (int64_t)npass_of(units[u].board) * units[u].cost >= a.hi_thr;
            if (hi == (pass == 0)) init_out[k++] = u;
        }
}

void build_units(const gol_board *h, int bindex, int K, int tile_rows, std::vector<UnitDesc> &units,
                 int32_t *nunits_out) {
    const UnitGrid g = unit_grid(h->srows, h->swords, K, tile_rows);
    const size_t first = units.size();
    units.resize(first + (size_t)g.nb * g.nt);
    // a tiled torus with a partial last word: that word and word 0 in the
    // middle of tile 0 (a halo word must hold K valid columns beyond the
    // tile, the partial word may hold fewer)
    const int seam = (h->masked && h->torus && !g.full) ? (int)(h->swords / g.nt) / 2 : 0;
    fill_units(h->srows, h->swords, bindex, g, units.data() + first, (int)first, seam);
    set_board_cost(units.data() + first, g.nb * g.nt, K);
    *nunits_out = g.nb * g.nt;
}

// Fraction of the lane work of a pass that produces cells: lanes holding
// words of the board (segments of full rows, or 30-word tiles) times the
// share of stage rows that are not halo recomputation.
double lane_efficiency(int64_t rows, int64_t words, int K, int tile_rows) {
    const UnitGrid g = unit_grid(rows, words, K, tile_rows);
    double useful = 0, work = 0;
    for (int i = 0; i < g.nb; ++i) {
        const int64_t bh = rows * (i + 1) / g.nb - rows * i / g.nb;
        const int64_t h = g.full ? (bh + g.S - 1) / g.S : bh;
        useful += (double)bh * words * K;
        work += 32.0 * g.nt * ((double)h * K + (double)K * (K - 1));
    }
    return work > 0 ? useful / work : 0;
}

// Tile rows of a board with `npass` passes under a chain cap (see build_plan).
// `chain_cap` bounds npass * H, the rows one unit streams through in all its
// passes (halo rows left out), so that no board's chain of passes outlasts
// the others' work.
int capped_tile_rows(int rows, int64_t npass, int K, double chain_cap) {
    if ((double)npass * rows > chain_cap) {
        const int h = (int)(chain_cap / (double)npass);
        rows = std::max(std::max(8, K), std::min(rows, h));
    }
    return rows;
}

// Chain cap as a fraction of the average work per warp slot.  With one board
// every unit has the same chain and the cap only sets the units per warp
// (measured best near 0.7 on a 16384^2 board); with many boards of uneven
// length a tighter cap keeps the longest chains off the critical path
// (measured best near 0.5 on the 4096-board batch).
double chain_fraction(size_t nboards) {
    if (g_opt_chain > 0) return (double)g_opt_chain / 1000.0;
    return nboards == 1 ? 0.7 : 0.5;
}

// Halo-free row iterations of all passes of a board's units: each warp lane
// segment streams ceil(R / S) rows per pass, for each of nt tiles.
double board_row_work(int64_t srows, int64_t swords, int64_t npass) {
    const int64_t S = swords <= 32 ? std::max<int64_t>(1, 32 / swords) : 1;
    const int64_t nt = swords <= 32 ? 1 : (swords + kTileWords - 1) / kTileWords;
    return (double)npass * (double)((srows + S - 1) / S) * (double)nt;
}

// Passes of board i in a launch: its generations in passes of at most K,
// or, in a population trace, each sampling period of `every` generations in
// ceil(every / K) passes.
int64_t plan_npass(const Plan &P, size_t i) {
    if (P.every > 0) return (P.gens[i] / P.every) * ((P.every + P.K - 1) / P.K);
    return (P.gens[i] + P.K - 1) / P.K;
}

int build_plan(Plan &P) {
    const size_t n = P.hs.size();
    P.boards.clear();
    P.units.clear();
    P.npass.clear();
    // one K per launch: the tuned K of the board with the most work
    int64_t best_work = -1;
    int K = 8;
    for (size_t i = 0; i < n; ++i) {
        const int64_t work = P.hs[i]->rows * P.hs[i]->cols * P.gens[i];
        if (work > best_work) {
            best_work = work;
            K = tune_lookup(P.hs[i]->srows, P.hs[i]->swords * 64).k;
        }
    }
    P.K = supported_k(std::max(1, K));
    // boards with a masked last word and population traces run kernel
    // variants 4 / 5 / 6, which exist for 4, 6 and 8 generations per pass
    P.masked = P.hs[0]->masked != 0;
    if (P.masked || P.every > 0) P.K = P.K >= 8 ? 8 : (P.K >= 6 ? 6 : 4);
    int64_t units_estimate = 0;    // with the tuned tile rows, before any chain cap
    for (size_t i = 0; i < n; ++i) {
        const UnitGrid ug = unit_grid(P.hs[i]->srows, P.hs[i]->swords, P.K,
                                      std::max(1, tune_lookup(P.hs[i]->srows, P.hs[i]->swords * 64).rows));
        units_estimate += (int64_t)ug.nb * ug.nt;
    }
    P.variant = P.masked ? (P.every > 0 ? 6 : 4) : (P.every > 0 ? 5 : plan_variant(P.K, units_estimate));
    int bps = 1;
    cudaError_t e = occupancy_for(P.K, P.torus, P.variant, &bps);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    const int64_t slots = (int64_t)g_dev.sms * std::max(1, bps) * kWarpsPerBlock;
    // Tile rows per board.  The tune table gives the tallest (most efficient)
    // unit; a board with many passes gets shorter units when its chain of
    // passes would exceed a fraction (GOL_OPT_CHAIN_PERMILLE) of the average
    // work per warp slot, so that long runs do not set the makespan and a
    // single board is split into enough units for every warp.
    std::vector<int> hrows(n);
    double work = 0;
    for (size_t i = 0; i < n; ++i) {
        const gol_board *h = P.hs[i];
        hrows[i] = std::max(1, tune_lookup(h->srows, h->swords * 64).rows);
        work += board_row_work(h->srows, h->swords, plan_npass(P, i));
    }
    const double chain_cap = g_opt_rows ? 1e300 : chain_fraction(n) * work / (double)slots;
    for (size_t i = 0; i < n; ++i)
        hrows[i] = capped_tile_rows(hrows[i], plan_npass(P, i), P.K, chain_cap);
    P.total_tasks = 0;
    P.boards.resize(n);
    P.npass.resize(n);
    // Units are numbered, and so queued at launch, longest chain of passes
    // first (npass * H): the boards that finish last start first.
    std::vector<size_t> order(n);
    for (size_t i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
        const double cx = (double)plan_npass(P, x) * hrows[x];
        const double cy = (double)plan_npass(P, y) * hrows[y];
        return cx > cy;
    });
    for (size_t i : order) {
        gol_board *h = P.hs[i];
        BoardDesc bd{};
        bd.buf[0] = (uint64_t *)h->buf[0];
        bd.buf[1] = (uint64_t *)h->buf[1];
        bd.cur = h->dev_cur;
        bd.R = (int32_t)h->srows;
        bd.W = (int32_t)h->swords;
        bd.gens = (int32_t)P.gens[i];
        bd.npass = (int32_t)plan_npass(P, i);
        bd.ppp = P.every > 0 ? (int32_t)((P.every + P.K - 1) / P.K) : 0;
        bd.pop_off = P.every > 0 ? P.pop_first[i] : 0;
        bd.last_bits = h->last_bits;
        build_units(h, (int)i, P.K, hrows[i], P.units, &bd.nunits);
        P.total_tasks += (int64_t)bd.nunits * bd.npass;
        P.boards[i] = bd;
        P.npass[i] = bd.npass;
    }
    if (P.total_tasks >= (int64_t(1) << 31) || P.units.size() >= (size_t(1) << 30))
        return fail(GOL_EINVAL, "batch too large for one launch (%lld tasks)", (long long)P.total_tasks);
    const size_t nb = P.boards.size(), nu = P.units.size();
    const int64_t max_blocks = (int64_t)g_dev.sms * std::max(1, bps);
    PersistArgs &a = P.args;
    P.init_order.resize(nu);
    plan_rings(P.units.data(), (int)nu, nb, [&](int b) { return P.boards[b].npass; }, a, P.init_order.data());
    // device memory: boards | units | init_order | run | next_pass | join | ctr | qctr | ring
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t o_units = al(nb * sizeof(BoardDesc));
    const size_t o_init = o_units + al(nu * sizeof(UnitDesc));
    const size_t o_run = o_init + al(nu * 4);
    const size_t o_next = o_run + al(nu * sizeof(UnitRun));
    const size_t o_join = o_next + al(nu * 4);
    const size_t o_ctr = o_join + al(2 * nu * 4);
    const size_t o_qctr = o_ctr + al((4 + nb) * 4);
    const size_t o_ring = o_qctr + al(32 * 4);
    P.dbytes = o_ring + al((size_t)P.total_tasks * 4);
    P.dmem = dev_alloc(P.dbytes, g_alloc, g_alloc_ctx);
    P.free_fn = g_free;
    P.alloc_ctx = g_alloc_ctx;
    if (!P.dmem) return fail(GOL_ENOMEM, "plan workspace of %zu bytes", P.dbytes);
    char *base = (char *)P.dmem;
    CU(upload({{base, P.boards.data(), nb * sizeof(BoardDesc)},
                {base + o_units, P.units.data(), nu * sizeof(UnitDesc)},
                {base + o_init, P.init_order.data(), nu * 4}}));
    a.boards = (const BoardDesc *)base;
    a.units = (const UnitDesc *)(base + o_units);
    a.run = (UnitRun *)(base + o_run);
    a.next_pass = (int32_t *)(base + o_next);
    a.join = (int32_t *)(base + o_join);
    a.ctr = (int32_t *)(base + o_ctr);
    a.qctr = (int32_t *)(base + o_qctr);
    a.init_order = (const int32_t *)(base + o_init);
    a.ring = (int32_t *)(base + o_ring);
    a.sticky = g_dev.sticky;
    a.nunits = (int32_t)nu;
    a.total_tasks = (int32_t)P.total_tasks;
    a.timeout_ns = g_opt_timeout_ms * 1000000ll;
    const int64_t want = (int64_t)(nu + kWarpsPerBlock - 1) / kWarpsPerBlock;
    P.grid = (int)std::max<int64_t>(1, std::min(max_blocks, want));
    a.nwarps = P.grid * kWarpsPerBlock;
    a.pad = 0;
    return GOL_OK;
}

cudaError_t launch_plan_kernels(const Plan &P, cudaStream_t s) {
    cudaError_t e = launch_sched_init(P.args, (int)P.boards.size(), s);
    if (e != cudaSuccess) return e;
    return launch_for(P.K, P.args, P.torus, P.variant, P.grid, s);
}

// plan cache (most recently used first); evicted plans wait in the
// graveyard until the work queued before their eviction has finished
// Both lists live on the heap and are never destroyed: at process exit the
// allocator hook (e.g. a Python callback) may already be gone, so no plan
// memory is released from a static destructor.
std::vector<std::unique_ptr<Plan>> &g_plans = *new std::vector<std::unique_ptr<Plan>>();
constexpr size_t kMaxPlans = 16;
struct Grave {
    std::unique_ptr<Plan> plan;
    cudaEvent_t ev;
};
std::vector<Grave> &g_graves = *new std::vector<Grave>();

void bury(std::unique_ptr<Plan> p) {
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ev, g_stream) != cudaSuccess) {
        cudaGetLastError();
        if (ev) cudaEventDestroy(ev);
        cudaDeviceSynchronize();
        return;   // plan freed now, after the device went idle
    }
    g_graves.push_back(Grave{std::move(p), ev});
}

void reap(bool all) {
    for (size_t i = 0; i < g_graves.size();) {
        if (all) cudaEventSynchronize(g_graves[i].ev);
        if (cudaEventQuery(g_graves[i].ev) == cudaSuccess) {
            cudaEventDestroy(g_graves[i].ev);
            g_graves.erase(g_graves.begin() + i);
        } else {
            cudaGetLastError();
            ++i;
        }
    }
}

// Boards destroyed while work queued before gol_destroy may still use them:
// their memory is freed once an event recorded at destruction has completed
// (never from a static destructor, like the plans).
struct BoardGrave {
    void *mem[3];
    void (*free_fn)(void *, void *);
    void *alloc_ctx;
    cudaGraphExec_t graphs[2];
    cudaEvent_t ev;
};
std::vector<BoardGrave> &g_board_graves = *new std::vector<BoardGrave>();

void free_board_memory(BoardGrave &g) {
    for (auto ge : g.graphs)
        if (ge) cudaGraphExecDestroy(ge);
    for (void *p : g.mem) dev_free(p, g.free_fn, g.alloc_ctx);
}

void reap_boards(bool all) {
    for (size_t i = 0; i < g_board_graves.size();) {
        if (all) cudaEventSynchronize(g_board_graves[i].ev);
        if (cudaEventQuery(g_board_graves[i].ev) == cudaSuccess) {
            free_board_memory(g_board_graves[i]);
            cudaEventDestroy(g_board_graves[i].ev);
            g_board_graves.erase(g_board_graves.begin() + i);
        } else {
            cudaGetLastError();
            ++i;
        }
    }
}

// Frees p once the work queued so far on the library's stream has run.
void defer_free(void *p, void (*ff)(void *, void *), void *ctx) {
    if (!p) return;
    BoardGrave g{{p, nullptr, nullptr}, ff, ctx, {nullptr, nullptr}, nullptr};
    if (cudaEventCreateWithFlags(&g.ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(g.ev, g_stream) != cudaSuccess) {
        cudaGetLastError();
        if (g.ev) cudaEventDestroy(g.ev);
        cudaStreamSynchronize(g_stream);
        free_board_memory(g);
        return;
    }
    g_board_graves.push_back(g);
}

void clear_plans() {
    for (auto &p : g_plans) bury(std::move(p));
    g_plans.clear();
    reap(true);
    reap_boards(true);
}

Plan *find_plan(const std::vector<gol_handle> &hs, const std::vector<int64_t> &gens, bool torus) {
    for (size_t i = 0; i < g_plans.size(); ++i) {
        Plan &P = *g_plans[i];
        if (P.torus != torus || P.hs.size() != hs.size() || P.opt_k != g_opt_k || P.opt_rows != g_opt_rows ||
            P.opt_chain != g_opt_chain || P.opt_variant != g_opt_variant || P.opt_critical != g_opt_critical)
            continue;
        if (P.gens != gens || P.hs != hs) continue;
        bool same = true;
        for (size_t j = 0; j < hs.size() && same; ++j) same = P.serials[j] == hs[j]->serial;
        if (!same) continue;
        if (P.args.timeout_ns != g_opt_timeout_ms * 1000000ll) continue;
        if (i) std::rotate(g_plans.begin(), g_plans.begin() + i, g_plans.begin() + i + 1);
        return g_plans[0].get();
    }
    return nullptr;
}

void drop_plans_of(gol_handle h) {
    for (size_t i = 0; i < g_plans.size();) {
        if (std::find(g_plans[i]->hs.begin(), g_plans[i]->hs.end(), h) != g_plans[i]->hs.end()) {
            bury(std::move(g_plans[i]));
            g_plans.erase(g_plans.begin() + i);
        } else {
            ++i;
        }
    }
}

// run packed boards (all with the same torus flag) in one persistent launch
int run_packed(const std::vector<gol_handle> &hs, const std::vector<int64_t> &gens, bool torus) {
    if (hs.empty()) return GOL_OK;
    Plan *P = find_plan(hs, gens, torus);
    if (!P) {
        auto np = std::make_unique<Plan>();
        np->hs = hs;
        np->gens = gens;
        np->torus = torus;
        np->opt_k = g_opt_k;
        np->opt_rows = g_opt_rows;
        np->opt_chain = g_opt_chain;
        np->opt_variant = g_opt_variant;
        np->opt_critical = g_opt_critical;

        for (auto h : hs) np->serials.push_back(h->serial);
        int rc = build_plan(*np);
        if (rc) return rc;
        reap(false);
        g_plans.insert(g_plans.begin(), std::move(np));
        if (g_plans.size() > kMaxPlans) {
            bury(std::move(g_plans.back()));
            g_plans.pop_back();
        }
        P = g_plans[0].get();
    }
    P->uses++;
    cudaError_t e;
    // replays of a repeated batch go through a CUDA graph (not on the legacy stream)
    if (g_opt_graphs && g_stream != nullptr && P->uses >= 2 && !P->no_graph) {
        if (!P->graph || P->graph_stream != g_stream) {
            if (P->graph) {
                cudaGraphExecDestroy(P->graph);
                P->graph = nullptr;
            }
            cudaGraph_t graph = nullptr;
            CU(cudaStreamBeginCapture(g_stream, cudaStreamCaptureModeThreadLocal));
            set_capturing(true);
            e = launch_plan_kernels(*P, g_stream);
            set_capturing(false);
            cudaError_t e2 = cudaStreamEndCapture(g_stream, &graph);
            if (e == cudaSuccess && e2 == cudaSuccess) {
                e = cudaGraphInstantiate(&P->graph, graph, 0);
                if (e != cudaSuccess) P->graph = nullptr;
            }
            if (graph) cudaGraphDestroy(graph);
            if (e != cudaSuccess || e2 != cudaSuccess || !P->graph) {
                // this launch cannot be captured here: launch it directly from now on
                cudaGetLastError();
                P->no_graph = true;
            } else {
                P->graph_stream = g_stream;
            }
        }
    }
    if (P->graph && !P->no_graph && g_opt_graphs && g_stream != nullptr && P->graph_stream == g_stream) {
        e = cudaGraphLaunch(P->graph, g_stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
        count_launches(2);   // the scheduler initialisation and the step kernel
    } else {
        e = launch_plan_kernels(*P, g_stream);
        if (e != cudaSuccess) return cuda_fail(e, "launching the step");
    }
    for (size_t i = 0; i < hs.size(); ++i) {
        hs[i]->cur ^= (P->npass[i] & 1);
        hs[i]->generation += gens[i];
    }
    return GOL_OK;
}

// Byte boards: one launch per generation.  Long runs on a non-default stream
// replay a captured CUDA graph of kByteGraphGens launches (an even number,
// so the current buffer is the same before and after a replay); one graph per
// starting buffer is kept with the board.
constexpr int kByteGraphGens = 64;

// Boards that fit the shared memory of one thread-block cluster run all
// their generations inside one launch (at most this many per launch).
constexpr int kByteClusterGensPerLaunch = 1 << 14;

int step_bytes(gol_handle h, int64_t G) {
    if (g_opt_byte_cluster && G > 0 && byte_cluster_size(h->rows, h->cols) > 0) {
        while (G > 0) {
            const int g = (int)std::min<int64_t>(G, kByteClusterGensPerLaunch);
            cudaError_t e = launch_byte_cluster((const uint8_t *)h->buf[h->cur], (uint8_t *)h->buf[h->cur ^ 1], h->rows,
                                                h->cols, h->torus, g, (int)g_opt_byte_cluster, g_stream);
            if (e != cudaSuccess) return cuda_fail(e, "byte cluster launch");
            h->cur ^= 1;
            h->generation += g;
            G -= g;
        }
        return GOL_OK;
    }
    if (g_opt_graphs && g_stream != nullptr && G >= 2 * kByteGraphGens) {
        if (h->byte_graph_stream != g_stream) {
            for (auto &ge : h->byte_graph)
                if (ge) {
                    cudaGraphExecDestroy(ge);
                    ge = nullptr;
                }
            h->byte_graph_stream = g_stream;
        }
        cudaGraphExec_t &ge = h->byte_graph[h->cur];
        if (!ge) {
            cudaGraph_t graph = nullptr;
            CU(cudaStreamBeginCapture(g_stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaSuccess;
            set_capturing(true);
            for (int g = 0; g < kByteGraphGens && e == cudaSuccess; ++g) {
                const int c = h->cur ^ (g & 1);
                e = launch_byte_step((const uint8_t *)h->buf[c], (uint8_t *)h->buf[c ^ 1], h->rows, h->cols,
                                     h->torus, g_stream);
            }
            set_capturing(false);
            cudaError_t e2 = cudaStreamEndCapture(g_stream, &graph);
            if (e != cudaSuccess) return cuda_fail(e, "capturing byte steps");
            if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&ge, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        }
        for (; G >= kByteGraphGens; G -= kByteGraphGens) {
            CU(cudaGraphLaunch(ge, g_stream));
            count_launches(kByteGraphGens);
            h->generation += kByteGraphGens;
        }
    }
    for (int64_t g = 0; g < G; ++g) {
        const uint8_t *in = (const uint8_t *)h->buf[h->cur];
        uint8_t *out = (uint8_t *)h->buf[h->cur ^ 1];
        cudaError_t e = launch_byte_step(in, out, h->rows, h->cols, h->torus, g_stream);
        if (e != cudaSuccess) return cuda_fail(e, "byte step launch");
        h->cur ^= 1;
        h->generation += 1;
    }
    return GOL_OK;
}

int set_cur_device(gol_handle h) {
    CU(cudaMemcpyAsync(h->dev_cur, &h->cur, sizeof(int32_t), cudaMemcpyHostToDevice, g_stream));
    return GOL_OK;
}

// split generation counts so that one launch stays within int32 task counts
constexpr int64_t kMaxGensPerLaunch = int64_t(1) << 24;

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *gol_last_error(void) { return t_err.c_str(); }

int gol_set_stream(void *s) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_stream = (cudaStream_t)s;
    return GOL_OK;
}

int gol_set_allocator(void *(*af)(size_t, void *), void (*ff)(void *, void *), void *ctx) {
    std::lock_guard<std::mutex> lk(g_mu);
    if ((af == nullptr) != (ff == nullptr)) return fail(GOL_EINVAL, "alloc and free must both be set or both null");
    clear_plans();
    g_alloc = af;
    g_free = ff;
    g_alloc_ctx = ctx;
    return GOL_OK;
}

int gol_create_ex(int64_t rows, int64_t cols, int torus, int layout, gol_handle *out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!out) return fail(GOL_EINVAL, "null output handle");
    *out = nullptr;
    if (rows < 1 || cols < 1) return fail(GOL_EINVAL, "rows and cols must be >= 1 (got %lld x %lld)",
                                          (long long)rows, (long long)cols);
    // a board with neither side a multiple of 64 is bytes when its cells fit
    // one thread-block cluster (all generations in one launch), else packed
    // with a masked last word
    if (layout == GOL_LAYOUT_AUTO)
        layout = (cols % 64 == 0 || rows % 64 == 0 || byte_cluster_size(rows, cols) == 0) ? GOL_LAYOUT_PACKED
                                                                                         : GOL_LAYOUT_BYTES;
    if (layout != GOL_LAYOUT_PACKED && layout != GOL_LAYOUT_BYTES) return fail(GOL_EINVAL, "unknown layout %d", layout);
    if (layout == GOL_LAYOUT_PACKED && (rows > (int64_t(1) << 30) || cols > (int64_t(1) << 30)))
        return fail(GOL_EINVAL, "board too large");
    int rc = ensure_device();
    if (rc) return rc;
    reap_boards(false);
    auto h = new gol_board();
    h->rows = rows;
    h->cols = cols;
    h->torus = torus ? 1 : 0;
    h->layout = layout;
    h->masked = layout == GOL_LAYOUT_PACKED && cols % 64 != 0 && rows % 64 != 0;
    h->last_bits = h->masked ? (int)(cols % 64) : 0;
    h->odd_width = layout == GOL_LAYOUT_PACKED && cols % 64 != 0 && !h->masked;
    h->words = layout == GOL_LAYOUT_PACKED && !h->odd_width ? (cols + 63) / 64 : 0;
    h->buf_bytes = layout == GOL_LAYOUT_PACKED ? (h->masked ? (size_t)rows * (size_t)h->words * 8
                                                            : (size_t)rows * (size_t)cols / 8)
                                               : (size_t)rows * (size_t)cols;
    h->alloc_fn = g_alloc;
    h->free_fn = g_free;
    h->alloc_ctx = g_alloc_ctx;
    h->serial = ++g_serial;
    h->srows = rows;
    h->swords = h->words;
    if (h->odd_width) {
        h->transposed = 1;
        h->srows = cols;
        h->swords = rows / 64;
    } else if (layout == GOL_LAYOUT_PACKED && !h->masked && rows % 64 == 0 && g_opt_orient != 1) {
        bool t = g_opt_orient == 2;
        if (!t) {
            const TuneEntry a = tune_lookup(rows, cols), b = tune_lookup(cols, rows);
            const double ea = lane_efficiency(rows, cols / 64, supported_k(a.k), a.rows);
            const double eb = lane_efficiency(cols, rows / 64, supported_k(b.k), b.rows);
            t = eb > 1.02 * ea;
        }
        if (t) {
            h->transposed = 1;
            h->srows = cols;
            h->swords = rows / 64;
        }
    }
    h->buf[0] = dev_alloc(h->buf_bytes, h->alloc_fn, h->alloc_ctx);
    h->buf[1] = dev_alloc(h->buf_bytes, h->alloc_fn, h->alloc_ctx);
    h->dev_cur = (int32_t *)dev_alloc(256, h->alloc_fn, h->alloc_ctx);
    if (!h->buf[0] || !h->buf[1] || !h->dev_cur) {
        dev_free(h->buf[0], h->free_fn, h->alloc_ctx);
        dev_free(h->buf[1], h->free_fn, h->alloc_ctx);
        dev_free(h->dev_cur, h->free_fn, h->alloc_ctx);
        delete h;
        return fail(GOL_ENOMEM, "could not allocate 2 x %zu bytes of device memory", (size_t)rows * cols);
    }
    cudaError_t e1 = cudaMemsetAsync(h->buf[0], 0, h->buf_bytes, g_stream);
    cudaError_t e2 = cudaMemsetAsync(h->buf[1], 0, h->buf_bytes, g_stream);
    cudaError_t e3 = cudaMemsetAsync(h->dev_cur, 0, 256, g_stream);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        dev_free(h->buf[0], h->free_fn, h->alloc_ctx);
        dev_free(h->buf[1], h->free_fn, h->alloc_ctx);
        dev_free(h->dev_cur, h->free_fn, h->alloc_ctx);
        delete h;
        return cuda_fail(e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3), "clearing a new board");
    }
    *out = h;
    return GOL_OK;
}

int gol_create(int64_t rows, int64_t cols, int torus, gol_handle *out) {
    return gol_create_ex(rows, cols, torus, GOL_LAYOUT_AUTO, out);
}

int gol_destroy(gol_handle h) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!valid(h)) return fail(GOL_EINVAL, "invalid handle");
    drop_plans_of(h);
    reap_boards(false);
    BoardGrave g{{h->buf[0], h->buf[1], h->dev_cur}, h->free_fn, h->alloc_ctx,
                 {h->byte_graph[0], h->byte_graph[1]}, nullptr};
    h->rows = 0;
    delete h;
    // the memory is freed once the work queued so far on the stream has run
    if (cudaEventCreateWithFlags(&g.ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(g.ev, g_stream) != cudaSuccess) {
        cudaGetLastError();
        if (g.ev) cudaEventDestroy(g.ev);
        cudaStreamSynchronize(g_stream);
        free_board_memory(g);
        return GOL_OK;
    }
    g_board_graves.push_back(g);
    return GOL_OK;
}

int gol_info(gol_handle h, int64_t *rows, int64_t *cols, int *torus, int *layout) {
    if (!valid(h)) return fail(GOL_EINVAL, "invalid handle");
    if (rows) *rows = h->rows;
    if (cols) *cols = h->cols;
    if (torus) *torus = h->torus;
    if (layout) *layout = h->layout;
    return GOL_OK;
}

int gol_set(gol_handle h, const uint8_t *cells, size_t n) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!valid(h) || !cells) return fail(GOL_EINVAL, "invalid handle or null cells");
    if (n != (size_t)h->rows * (size_t)h->cols)
        return fail(GOL_EINVAL, "n = %zu, board has %lld cells", n, (long long)(h->rows * h->cols));
    for (size_t i = 0; i < n; ++i)
        if (cells[i] > 1) return fail(GOL_EINVAL, "cell %zu has value %u (must be 0 or 1)", i, (unsigned)cells[i]);
    h->cur = 0;
    h->generation = 0;
    if (h->layout == GOL_LAYOUT_BYTES) {
        CU(cudaMemcpyAsync(h->buf[0], cells, n, cudaMemcpyHostToDevice, g_stream));
    } else {
        const size_t flag_off = (n + 255) & ~size_t(255);
        Scratch st(flag_off + 256);
        if (!st.p) return fail(GOL_ENOMEM, "staging buffer of %zu bytes", n);
        int32_t *bad = (int32_t *)((char *)st.p + flag_off);
        CU(cudaMemsetAsync(bad, 0, sizeof(int32_t), g_stream));
        CU(cudaMemcpyAsync(st.p, cells, n, cudaMemcpyHostToDevice, g_stream));
        if (h->odd_width) {
            CU(launch_pack_transposed((const uint8_t *)st.p, h->rows, h->cols, (uint64_t *)h->buf[0], bad, g_stream));
        } else if (h->masked) {
            CU(launch_pack_rows((const uint8_t *)st.p, (uint64_t *)h->buf[1], h->rows, h->cols, bad, g_stream));
            CU(launch_orient((const uint64_t *)h->buf[1], (uint64_t *)h->buf[0], h->rows, h->words, false, true,
                             g_stream, h->last_bits));
        } else {
            CU(launch_pack((const uint8_t *)st.p, (uint64_t *)h->buf[1], h->rows, h->words, bad, g_stream));
            CU(launch_orient((const uint64_t *)h->buf[1], (uint64_t *)h->buf[0], h->rows, h->words, h->transposed,
                             true, g_stream));
        }
        int32_t bad_h = 0;
        CU(cudaMemcpyAsync(&bad_h, bad, sizeof bad_h, cudaMemcpyDeviceToHost, g_stream));
        CU(cudaStreamSynchronize(g_stream));
        if (bad_h) return fail(GOL_EINVAL, "cell values other than 0/1 reached the device");
    }
    int rc = set_cur_device(h);
    if (rc) return rc;
    return sync_stream();
}

int gol_get(gol_handle h, uint8_t *cells, size_t n) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!valid(h) || !cells) return fail(GOL_EINVAL, "invalid handle or null cells");
    if (n != (size_t)h->rows * (size_t)h->cols)
        return fail(GOL_EINVAL, "n = %zu, board has %lld cells", n, (long long)(h->rows * h->cols));
    if (h->layout == GOL_LAYOUT_BYTES) {
        CU(cudaMemcpyAsync(cells, h->buf[h->cur], n, cudaMemcpyDeviceToHost, g_stream));
        return sync_stream();
    }
    const size_t woff = (n + 255) & ~size_t(255);
    Scratch st(woff + (size_t)h->rows * (size_t)((h->cols + 63) / 64) * 8);
    if (!st.p) return fail(GOL_ENOMEM, "staging buffer of %zu bytes", n);
    if (h->odd_width) {
        CU(launch_unpack_transposed((const uint64_t *)h->buf[h->cur], h->rows, h->cols, (uint8_t *)st.p, g_stream));
    } else if (h->masked) {
        uint64_t *words = (uint64_t *)((char *)st.p + woff);
        CU(launch_orient((const uint64_t *)h->buf[h->cur], words, h->rows, h->words, false, false, g_stream,
                         h->last_bits));
        CU(launch_unpack_rows(words, (uint8_t *)st.p, h->rows, h->cols, g_stream));
    } else {
        uint64_t *words = (uint64_t *)((char *)st.p + woff);
        CU(launch_orient((const uint64_t *)h->buf[h->cur], words, h->rows, h->words, h->transposed, false,
                         g_stream));
        CU(launch_unpack(words, (uint8_t *)st.p, h->rows, h->words, g_stream));
    }
    CU(cudaMemcpyAsync(cells, st.p, n, cudaMemcpyDeviceToHost, g_stream));
    return sync_stream();
}

int gol_set_packed(gol_handle h, const uint64_t *words, size_t nwords) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!valid(h) || !words) return fail(GOL_EINVAL, "invalid handle or null words");
    if (h->layout != GOL_LAYOUT_PACKED) return fail(GOL_EINVAL, "board is not packed");
    if (h->odd_width) return fail(GOL_EINVAL, "a board %lld cells wide has no packed word layout", (long long)h->cols);
    if (nwords != (size_t)(h->rows * h->words))
        return fail(GOL_EINVAL, "nwords = %zu, board has %lld words", nwords, (long long)(h->rows * h->words));
    h->cur = 0;
    h->generation = 0;
    CU(cudaMemcpyAsync(h->buf[1], words, nwords * 8, cudaMemcpyHostToDevice, g_stream));
    CU(launch_orient((const uint64_t *)h->buf[1], (uint64_t *)h->buf[0], h->rows, h->words, h->transposed, true,
                     g_stream, h->last_bits));
    return set_cur_device(h);
}

int gol_get_packed(gol_handle h, uint64_t *words, size_t nwords) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!valid(h) || !words) return fail(GOL_EINVAL, "invalid handle or null words");
    if (h->layout != GOL_LAYOUT_PACKED) return fail(GOL_EINVAL, "board is not packed");
    if (h->odd_width) return fail(GOL_EINVAL, "a board %lld cells wide has no packed word layout", (long long)h->cols);
    if (nwords != (size_t)(h->rows * h->words))
        return fail(GOL_EINVAL, "nwords = %zu, board has %lld words", nwords, (long long)(h->rows * h->words));
    Scratch st(nwords * 8);
    if (!st.p) return fail(GOL_ENOMEM, "staging buffer of %zu bytes", nwords * 8);
    CU(launch_orient((const uint64_t *)h->buf[h->cur], (uint64_t *)st.p, h->rows, h->words, h->transposed, false,
                     g_stream, h->last_bits));
    CU(cudaMemcpyAsync(words, st.p, nwords * 8, cudaMemcpyDeviceToHost, g_stream));
    return sync_stream();
}

int gol_set_packed_device(gol_handle h, const uint64_t *dwords, size_t nwords) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!valid(h) || !dwords) return fail(GOL_EINVAL, "invalid handle or null words");
    if (h->layout != GOL_LAYOUT_PACKED) return fail(GOL_EINVAL, "board is not packed");
    if (h->odd_width) return fail(GOL_EINVAL, "a board %lld cells wide has no packed word layout", (long long)h->cols);
    if (nwords != (size_t)(h->rows * h->words))
        return fail(GOL_EINVAL, "nwords = %zu, board has %lld words", nwords, (long long)(h->rows * h->words));
    h->cur = 0;
    h->generation = 0;
    if (dwords == h->buf[0] || dwords == h->buf[1]) return fail(GOL_EINVAL, "source is the board's own buffer");
    CU(launch_orient(dwords, (uint64_t *)h->buf[0], h->rows, h->words, h->transposed, true, g_stream,
                     h->last_bits));
    return set_cur_device(h);
}

int gol_get_packed_device(gol_handle h, uint64_t *dwords, size_t nwords) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!valid(h) || !dwords) return fail(GOL_EINVAL, "invalid handle or null words");
    if (h->layout != GOL_LAYOUT_PACKED) return fail(GOL_EINVAL, "board is not packed");
    if (h->odd_width) return fail(GOL_EINVAL, "a board %lld cells wide has no packed word layout", (long long)h->cols);
    if (nwords != (size_t)(h->rows * h->words))
        return fail(GOL_EINVAL, "nwords = %zu, board has %lld words", nwords, (long long)(h->rows * h->words));
    CU(launch_orient((const uint64_t *)h->buf[h->cur], dwords, h->rows, h->words, h->transposed, false, g_stream,
                     h->last_bits));
    return GOL_OK;
}

namespace {
// shared checks of the many-board transfers; fills descriptors and offsets
// Many-board transfer plans, cached by handle list (a batch moved every step
// reuses its plan): the boards' copy descriptors and the copy grid's
// block-to-board table, in device memory.  Descriptors name both buffers
// and the device `cur` of a board, so they stay valid while it is stepped.
struct CopyPlan {
    std::vector<gol_handle> hs;
    std::vector<uint64_t> serials;
    int64_t nwords = 0, blocks = 0;
    bool distinct = true;
    bool transposed = false;           // some board is stored transposed
    std::vector<CopyDesc> d;           // host copies of what dmem holds
    std::vector<int32_t> bb;
    void *dmem = nullptr;              // CopyDesc[n] | int32 block_board[blocks]
    size_t board_off = 0;
    void (*free_fn)(void *, void *) = nullptr;
    void *alloc_ctx = nullptr;
    const CopyDesc *desc() const { return (const CopyDesc *)dmem; }
    const int32_t *block_board() const { return (const int32_t *)((const char *)dmem + board_off); }
    ~CopyPlan() {
        if (dmem) {
            if (!free_fn) {
                cudaStreamSynchronize(g_stream);
                dev_free(dmem, free_fn, alloc_ctx);
            } else {
                defer_free(dmem, free_fn, alloc_ctx);
            }
        }
    }
};
// heap-allocated and never destroyed, like the step plans (see g_plans)
std::vector<std::unique_ptr<CopyPlan>> &g_copy_plans = *new std::vector<std::unique_ptr<CopyPlan>>();
constexpr size_t kMaxCopyPlans = 8;

int copy_plan(const gol_handle *hs, size_t n, const CopyPlan **out) {
    if (!hs) return fail(GOL_EINVAL, "null handle array");
    if (n > (size_t)(1 << 30)) return fail(GOL_EINVAL, "too many boards");
    for (size_t i = 0; i < n; ++i) {
        if (!valid(hs[i])) return fail(GOL_EINVAL, "invalid handle at %zu", i);
        if (hs[i]->layout != GOL_LAYOUT_PACKED) return fail(GOL_EINVAL, "board %zu is not packed", i);
        if (hs[i]->odd_width) return fail(GOL_EINVAL, "board %zu is %lld cells wide: no packed word layout", i,
                                          (long long)hs[i]->cols);
    }
    for (size_t k = 0; k < g_copy_plans.size(); ++k) {
        const CopyPlan &P = *g_copy_plans[k];
        if (P.hs.size() != n || !std::equal(hs, hs + n, P.hs.begin())) continue;
        bool same = true;
        for (size_t j = 0; j < n && same; ++j) same = P.serials[j] == hs[j]->serial;
        if (!same) continue;
        if (k) std::rotate(g_copy_plans.begin(), g_copy_plans.begin() + k, g_copy_plans.begin() + k + 1);
        *out = g_copy_plans[0].get();
        return GOL_OK;
    }
    auto P = std::make_unique<CopyPlan>();
    P->hs.assign(hs, hs + n);
    std::unordered_set<gol_handle> seen;
    std::vector<CopyDesc> &d = P->d;
    std::vector<int32_t> &bb = P->bb;
    d.resize(n);
    for (size_t i = 0; i < n; ++i) {
        gol_handle h = hs[i];
        P->serials.push_back(h->serial);
        if (!seen.insert(h).second) P->distinct = false;
        const int64_t nw = h->rows * h->words;
        d[i].buf[0] = (uint64_t *)h->buf[0];
        d[i].buf[1] = (uint64_t *)h->buf[1];
        d[i].cur = h->dev_cur;
        d[i].offset = P->nwords;
        d[i].nwords = nw;
        d[i].rows = h->rows;
        d[i].words = h->words;
        d[i].transposed = h->transposed;
        d[i].last_bits = h->last_bits;
        d[i].block0 = P->blocks;
        P->transposed = P->transposed || h->transposed;
        const int64_t nb = copy_blocks(d[i]);
        if (P->blocks + nb > INT32_MAX) return fail(GOL_EINVAL, "too many words in one transfer");
        bb.insert(bb.end(), (size_t)nb, (int32_t)i);
        P->blocks += nb;
        P->nwords += nw;
    }
    P->board_off = (n * sizeof(CopyDesc) + 255) & ~size_t(255);
    P->free_fn = g_free;
    P->alloc_ctx = g_alloc_ctx;
    P->dmem = dev_alloc(P->board_off + bb.size() * 4 + 4, g_alloc, g_alloc_ctx);
    if (!P->dmem) return fail(GOL_ENOMEM, "transfer plan of %zu boards", n);
    CU(upload({{P->dmem, d.data(), n * sizeof(CopyDesc)}, {(char *)P->dmem + P->board_off, bb.data(), bb.size() * 4}}));
    g_copy_plans.insert(g_copy_plans.begin(), std::move(P));
    if (g_copy_plans.size() > kMaxCopyPlans) g_copy_plans.pop_back();
    *out = g_copy_plans[0].get();
    return GOL_OK;
}
}  // namespace

namespace {
// The device address of page-locked host memory registered with CUDA
// (cudaHostAlloc, cudaHostRegister, a pinned torch tensor), which kernels on
// this GPU read and write in place over the chip-to-chip link; null for any
// other pointer (pageable memory goes through a staging buffer).  In place
// pays for transfers without boards stored transposed: a 32 MiB board moves
// in 0.18 / 0.21 ms up / down in place against 0.20 / 0.24 ms staged, a
// 2 GiB board in 10–20 ms each way (two runs) against 51.6 / 81.2 ms.  Tile transposes
// read and write 64-byte pieces of rows, which the copy engine plus a
// device-side pass moves faster (4096-board batch: 0.76 / 0.84 ms staged
// against 0.80 / 0.98 ms in place).
const void *mapped_host_pointer(const void *p, const CopyPlan &P) {
    if (!g_opt_zero_copy || P.transposed) return nullptr;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}
}  // namespace

int gol_set_packed_batch(const gol_handle *hs, size_t n, const uint64_t *words, size_t nwords) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (n == 0) return GOL_OK;
    if (!words) return fail(GOL_EINVAL, "null words");
    const CopyPlan *P = nullptr;
    int rc = copy_plan(hs, n, &P);
    if (rc) return rc;
    if (!P->distinct) return fail(GOL_EINVAL, "a handle is repeated");
    if ((int64_t)nwords != P->nwords)
        return fail(GOL_EINVAL, "nwords = %zu, the boards hold %lld words", nwords, (long long)P->nwords);
    const uint64_t *src = (const uint64_t *)mapped_host_pointer(words, *P);
    std::unique_ptr<Scratch> st;
    if (!src) {
        st.reset(new Scratch(nwords * 8));
        if (!st->p) return fail(GOL_ENOMEM, "staging buffer of %zu bytes", nwords * 8);
        CU(cudaMemcpyAsync(st->p, words, nwords * 8, cudaMemcpyHostToDevice, g_stream));
        src = (const uint64_t *)st->p;
    }
    CU(launch_scatter_boards(P->desc(), P->block_board(), P->blocks, src, g_stream));
    for (size_t i = 0; i < n; ++i) {
        hs[i]->cur = 0;
        hs[i]->generation = 0;
    }
    return GOL_OK;
}

int gol_get_packed_batch(const gol_handle *hs, size_t n, uint64_t *words, size_t nwords) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (n == 0) return GOL_OK;
    if (!words) return fail(GOL_EINVAL, "null words");
    const CopyPlan *P = nullptr;
    int rc = copy_plan(hs, n, &P);
    if (rc) return rc;
    if ((int64_t)nwords != P->nwords)
        return fail(GOL_EINVAL, "nwords = %zu, the boards hold %lld words", nwords, (long long)P->nwords);
    uint64_t *dst = (uint64_t *)mapped_host_pointer(words, *P);
    std::unique_ptr<Scratch> st;
    if (!dst) {
        st.reset(new Scratch(nwords * 8));
        if (!st->p) return fail(GOL_ENOMEM, "staging buffer of %zu bytes", nwords * 8);
    }
    CU(launch_gather_boards(P->desc(), P->block_board(), P->blocks, dst ? dst : (uint64_t *)st->p, g_stream));
    if (!dst) CU(cudaMemcpyAsync(words, st->p, nwords * 8, cudaMemcpyDeviceToHost, g_stream));
    return sync_stream();
}

int gol_get_packed_batch_async(const gol_handle *hs, size_t n, uint64_t *words, size_t nwords) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (n == 0) return GOL_OK;
    if (!words) return fail(GOL_EINVAL, "null words");
    const CopyPlan *P = nullptr;
    int rc = copy_plan(hs, n, &P);
    if (rc) return rc;
    if ((int64_t)nwords != P->nwords)
        return fail(GOL_EINVAL, "nwords = %zu, the boards hold %lld words", nwords, (long long)P->nwords);
    uint64_t *dst = (uint64_t *)mapped_host_pointer(words, *P);
    std::unique_ptr<Scratch> st;
    if (!dst) {
        st.reset(new Scratch(nwords * 8));
        if (!st->p) return fail(GOL_ENOMEM, "staging buffer of %zu bytes", nwords * 8);
    }
    CU(launch_gather_boards(P->desc(), P->block_board(), P->blocks, dst ? dst : (uint64_t *)st->p, g_stream));
    if (!dst) CU(cudaMemcpyAsync(words, st->p, nwords * 8, cudaMemcpyDeviceToHost, g_stream));
    return GOL_OK;
}

int gol_get_region(gol_handle h, int64_t r0, int64_t c0, int64_t nr, int64_t nc, uint8_t *out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!valid(h)) return fail(GOL_EINVAL, "invalid handle");
    if (nr < 0 || nc < 0) return fail(GOL_EINVAL, "negative window size");
    if (nr == 0 || nc == 0) return GOL_OK;
    if (!out) return fail(GOL_EINVAL, "null output");
    const size_t n = (size_t)nr * (size_t)nc;
    Scratch st(n);
    if (!st.p) return fail(GOL_ENOMEM, "staging buffer of %zu bytes", n);
    if (h->layout == GOL_LAYOUT_PACKED)
        CU(launch_region_packed((const uint64_t *)h->buf[h->cur], h->rows, h->cols, r0, c0, nr, nc,
                                (uint8_t *)st.p, h->transposed != 0, g_stream));
    else
        CU(launch_region_bytes((const uint8_t *)h->buf[h->cur], h->rows, h->cols, r0, c0, nr, nc,
                               (uint8_t *)st.p, g_stream));
    CU(cudaMemcpyAsync(out, st.p, n, cudaMemcpyDeviceToHost, g_stream));
    return sync_stream();
}

int gol_step(gol_handle h, int64_t generations) {
    gol_handle hs[1] = {h};
    int64_t gs[1] = {generations};
    return gol_step_batch(hs, gs, 1);
}

namespace {
int step_batch_locked(const gol_handle *hs, const int64_t *generations, size_t n);
}

int gol_step_batch(const gol_handle *hs, const int64_t *generations, size_t n) {
    std::lock_guard<std::mutex> lk(g_mu);
    return step_batch_locked(hs, generations, n);
}

namespace {
// One launch of a population trace: packed boards `hs` (one torus flag),
// board i advanced by gens[i], a whole number of periods of `every`
// generations; the step kernel adds the live cells of every unit at the end
// of each period into pop[pop_first[i] + period].  The plan is built for
// this launch alone (its sample slots are this call's) and freed once the
// launch has run.
int run_packed_trace(const std::vector<gol_handle> &hs, const std::vector<int64_t> &gens, bool torus, int64_t every,
                     const std::vector<int32_t> &pop_first, unsigned long long *pop) {
    auto P = std::make_unique<Plan>();
    P->hs = hs;
    P->gens = gens;
    P->torus = torus;
    P->every = every;
    P->pop_first = pop_first;
    for (auto h : hs) P->serials.push_back(h->serial);
    int rc = build_plan(*P);
    if (rc) return rc;
    P->args.pop = pop;
    cudaError_t e = launch_plan_kernels(*P, g_stream);
    if (e != cudaSuccess) return cuda_fail(e, "launching a population trace");
    for (size_t i = 0; i < hs.size(); ++i) {
        hs[i]->cur ^= (P->npass[i] & 1);
        hs[i]->generation += gens[i];
    }
    bury(std::move(P));
    return GOL_OK;
}

int step_batch_locked(const gol_handle *hs, const int64_t *generations, size_t n);

int population_trace_locked(const gol_handle *hs, size_t n, int64_t every, size_t samples, uint64_t *out) {
    if (n == 0 || samples == 0) return GOL_OK;
    if (!hs || !out) return fail(GOL_EINVAL, "null handles or output");
    if (every < 1) return fail(GOL_EINVAL, "every must be >= 1");
    if (samples > ((size_t)1 << 30) / n) return fail(GOL_EINVAL, "too many samples (%zu x %zu)", n, samples);
    const uint64_t stamp = ++g_batch_stamp;
    for (size_t i = 0; i < n; ++i) {
        if (!valid(hs[i])) return fail(GOL_EINVAL, "invalid handle at %zu", i);
        if (hs[i]->batch_stamp == stamp) return fail(GOL_EINVAL, "handle repeated at %zu", i);
        hs[i]->batch_stamp = stamp;
    }
    Scratch st(n * samples * sizeof(unsigned long long));
    if (!st.p) return fail(GOL_ENOMEM, "population trace slots");
    unsigned long long *slots = (unsigned long long *)st.p;
    CU(cudaMemsetAsync(slots, 0, n * samples * sizeof(unsigned long long), g_stream));
    // byte boards, and any board whose period is longer than one launch:
    // advanced and counted sample by sample
    for (size_t i = 0; i < n; ++i) {
        gol_handle h = hs[i];
        if (h->layout == GOL_LAYOUT_PACKED && every <= kMaxGensPerLaunch) continue;
        for (size_t k = 0; k < samples; ++k) {
            int rc = step_batch_locked(&h, &every, 1);
            if (rc) return rc;
            if (h->layout == GOL_LAYOUT_PACKED)
                CU(launch_popcount_packed((const uint64_t *)h->buf[h->cur], h->srows * h->swords,
                                          slots + i * samples + k, g_stream));
            else
                CU(launch_popcount_bytes((const uint8_t *)h->buf[h->cur], h->rows * h->cols,
                                         slots + i * samples + k, g_stream));
        }
    }
    // packed boards: counted inside the step kernel, one launch per torus
    // flag and run of whole periods
    if (every <= kMaxGensPerLaunch) {
        const size_t per = (size_t)std::max<int64_t>(1, kMaxGensPerLaunch / every);
        for (int group = 0; group < 4; ++group) {
            const int torus = group < 2 ? 1 : 0, masked = group & 1;
            std::vector<gol_handle> grp;
            std::vector<size_t> idx;
            for (size_t i = 0; i < n; ++i)
                if (hs[i]->layout == GOL_LAYOUT_PACKED && hs[i]->torus == torus && hs[i]->masked == masked) {
                    grp.push_back(hs[i]);
                    idx.push_back(i);
                }
            for (size_t s0 = 0; s0 < samples && !grp.empty(); s0 += per) {
                const size_t m = std::min(per, samples - s0);
                std::vector<int64_t> g(grp.size(), (int64_t)m * every);
                std::vector<int32_t> first(grp.size());
                for (size_t j = 0; j < grp.size(); ++j) first[j] = (int32_t)(idx[j] * samples + s0);
                int rc = run_packed_trace(grp, g, torus == 1, every, first, slots);
                if (rc) return rc;
            }
        }
    }
    CU(cudaMemcpyAsync(out, slots, n * samples * sizeof(unsigned long long), cudaMemcpyDeviceToHost, g_stream));
    return sync_stream();
}
}  // namespace

int gol_population_trace(gol_handle h, int64_t every, size_t n, uint64_t *out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!valid(h)) return fail(GOL_EINVAL, "invalid handle");
    return population_trace_locked(&h, 1, every, n, out);
}

int gol_population_trace_batch(const gol_handle *hs, size_t n, int64_t every, size_t samples, uint64_t *out) {
    std::lock_guard<std::mutex> lk(g_mu);
    return population_trace_locked(hs, n, every, samples, out);
}

namespace {
int step_batch_locked(const gol_handle *hs, const int64_t *generations, size_t n) {
    if (n == 0) return GOL_OK;
    if (!hs || !generations) return fail(GOL_EINVAL, "null arrays");
    // repeated handles: each call stamps the boards it lists (no per-call allocation)
    const uint64_t stamp = ++g_batch_stamp;
    for (size_t i = 0; i < n; ++i) {
        if (!valid(hs[i])) return fail(GOL_EINVAL, "invalid handle at %zu", i);
        if (generations[i] < 0) return fail(GOL_EINVAL, "negative generation count at %zu", i);
        if (hs[i]->batch_stamp == stamp) return fail(GOL_EINVAL, "handle repeated at %zu", i);
        hs[i]->batch_stamp = stamp;
    }
    // byte boards one by one
    for (size_t i = 0; i < n; ++i)
        if (hs[i]->layout == GOL_LAYOUT_BYTES && generations[i] > 0) {
            int rc = step_bytes(hs[i], generations[i]);
            if (rc) return rc;
        }
    // packed boards: torus and bounded groups, boards with and without a
    // masked last word apart, split into launches of at most
    // kMaxGensPerLaunch generations
    for (int group = 0; group < 4; ++group) {
        const int torus = group < 2 ? 1 : 0, masked = group & 1;
        std::vector<gol_handle> grp;
        std::vector<int64_t> left;
        for (size_t i = 0; i < n; ++i)
            if (hs[i]->layout == GOL_LAYOUT_PACKED && hs[i]->torus == torus && hs[i]->masked == masked &&
                generations[i] > 0) {
                grp.push_back(hs[i]);
                left.push_back(generations[i]);
            }
        while (!grp.empty()) {
            std::vector<gol_handle> now;
            std::vector<int64_t> g;
            for (size_t i = 0; i < grp.size(); ++i) {
                const int64_t take = std::min(left[i], kMaxGensPerLaunch);
                now.push_back(grp[i]);
                g.push_back(take);
                left[i] -= take;
            }
            int rc = run_packed(now, g, torus == 1);
            if (rc) return rc;
            std::vector<gol_handle> g2;
            std::vector<int64_t> l2;
            for (size_t i = 0; i < grp.size(); ++i)
                if (left[i] > 0) {
                    g2.push_back(grp[i]);
                    l2.push_back(left[i]);
                }
            grp.swap(g2);
            left.swap(l2);
        }
    }
    return GOL_OK;
}
}  // namespace

int gol_population(gol_handle h, uint64_t *out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!valid(h) || !out) return fail(GOL_EINVAL, "invalid handle or null output");
    Scratch st(sizeof(unsigned long long));
    if (!st.p) return fail(GOL_ENOMEM, "population scratch");
    CU(cudaMemsetAsync(st.p, 0, sizeof(unsigned long long), g_stream));
    if (h->layout == GOL_LAYOUT_PACKED)
        CU(launch_popcount_packed((const uint64_t *)h->buf[h->cur], h->srows * h->swords,
                                  (unsigned long long *)st.p, g_stream));
    else
        CU(launch_popcount_bytes((const uint8_t *)h->buf[h->cur], h->rows * h->cols,
                                 (unsigned long long *)st.p, g_stream));
    unsigned long long v = 0;
    CU(cudaMemcpyAsync(&v, st.p, sizeof v, cudaMemcpyDeviceToHost, g_stream));
    int rc = sync_stream();
    if (rc) return rc;
    *out = v;
    return GOL_OK;
}

int gol_generation(gol_handle h, int64_t *out) {
    if (!valid(h) || !out) return fail(GOL_EINVAL, "invalid handle or null output");
    *out = h->generation;
    return GOL_OK;
}

int gol_sync(gol_handle h) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!valid(h)) return fail(GOL_EINVAL, "invalid handle");
    return sync_stream();
}

int gol_set_option(int key, int64_t v) {
    std::lock_guard<std::mutex> lk(g_mu);
    switch (key) {
        case GOL_OPT_GENS_PER_PASS:
            if (!(v == 0 || is_supported_k((int)v)))
                return fail(GOL_EINVAL, "generations per pass must be 0 or one of 1, 2, 3, 4, 5, 6, 7, 8, 16");
            g_opt_k = v;
            return GOL_OK;
        case GOL_OPT_TILE_ROWS:
            if (v < 0 || v > (1 << 20)) return fail(GOL_EINVAL, "tile rows out of range");
            g_opt_rows = v;
            return GOL_OK;
        case GOL_OPT_USE_GRAPHS:
            g_opt_graphs = v ? 1 : 0;
            return GOL_OK;
        case GOL_OPT_WAIT_TIMEOUT_MS:
            if (v < 1 || v > 3600000) return fail(GOL_EINVAL, "timeout out of range");
            g_opt_timeout_ms = v;
            return GOL_OK;
        case GOL_OPT_ORIENTATION:
            if (v < 0 || v > 2) return fail(GOL_EINVAL, "orientation must be 0, 1 or 2");
            g_opt_orient = v;
            return GOL_OK;
        case GOL_OPT_CHAIN_PERMILLE:
            if (v < 0 || v > 100000) return fail(GOL_EINVAL, "chain fraction out of range");
            g_opt_chain = v;
            return GOL_OK;
        case GOL_OPT_PIPELINE:
            if (v < -1 || v > 3) return fail(GOL_EINVAL, "pipeline variant must be -1, 0, 1, 2 or 3");
            g_opt_variant = v;
            return GOL_OK;
        case GOL_OPT_ZERO_COPY:
            if (v < 0 || v > 1) return fail(GOL_EINVAL, "zero copy must be 0 or 1");
            g_opt_zero_copy = v;
            return GOL_OK;
        case GOL_OPT_BYTE_CLUSTER:
            if (v < 0 || v > 8 || (v > 1 && (v & (v - 1)))) return fail(GOL_EINVAL, "byte cluster must be 0, 1, 2, 4 or 8");
            g_opt_byte_cluster = v;
            return GOL_OK;
        case GOL_OPT_CRITICAL_PERMILLE:
            if (v < -1 || v > 1000) return fail(GOL_EINVAL, "critical permille must be -1 or in [0, 1000]");
            g_opt_critical = v;
            return GOL_OK;
    }
    return fail(GOL_EINVAL, "unknown option %d", key);
}

int gol_get_option(int key, int64_t *v) {
    if (!v) return fail(GOL_EINVAL, "null output");
    switch (key) {
        case GOL_OPT_GENS_PER_PASS: *v = g_opt_k; return GOL_OK;
        case GOL_OPT_TILE_ROWS: *v = g_opt_rows; return GOL_OK;
        case GOL_OPT_USE_GRAPHS: *v = g_opt_graphs; return GOL_OK;
        case GOL_OPT_WAIT_TIMEOUT_MS: *v = g_opt_timeout_ms; return GOL_OK;
        case GOL_OPT_ORIENTATION: *v = g_opt_orient; return GOL_OK;
        case GOL_OPT_CHAIN_PERMILLE: *v = g_opt_chain; return GOL_OK;
        case GOL_OPT_PIPELINE: *v = g_opt_variant; return GOL_OK;
        case GOL_OPT_ZERO_COPY: *v = g_opt_zero_copy; return GOL_OK;
        case GOL_OPT_BYTE_CLUSTER: *v = g_opt_byte_cluster; return GOL_OK;
        case GOL_OPT_CRITICAL_PERMILLE: *v = g_opt_critical; return GOL_OK;
    }
    return fail(GOL_EINVAL, "unknown option %d", key);
}

int gol_tune_set(int64_t rows, int64_t cols, int k, int tile_rows) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (rows < 1 || cols < 1 || !is_supported_k(k) || tile_rows < 1)
        return fail(GOL_EINVAL, "bad tune entry");
    g_tune[size_class(rows, cols)] = TuneEntry{k, tile_rows};
    clear_plans();
    return GOL_OK;
}

int gol_tune_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_tune.clear();
    clear_plans();
    return GOL_OK;
}

int gol_tune_get(int64_t rows, int64_t cols, int *k, int *tile_rows) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (rows < 1 || cols < 1) return fail(GOL_EINVAL, "bad size");
    TuneEntry t = tune_lookup(rows, cols);
    if (k) *k = supported_k(t.k);
    if (tile_rows) *tile_rows = t.rows;
    return GOL_OK;
}

int gol_tune_class(int64_t rows, int64_t cols, int *row_class, int *word_class) {
    if (rows < 1 || cols < 1) return fail(GOL_EINVAL, "bad size");
    const std::pair<int, int> c = size_class(rows, cols);
    if (row_class) *row_class = c.first;
    if (word_class) *word_class = c.second;
    return GOL_OK;
}

int gol_board_storage(gol_handle h, int64_t *srows, int64_t *swords, int *transposed) {
    if (!valid(h)) return fail(GOL_EINVAL, "invalid handle");
    const bool packed = h->layout == GOL_LAYOUT_PACKED;
    if (srows) *srows = packed ? h->srows : h->rows;
    if (swords) *swords = packed ? h->swords : 0;
    if (transposed) *transposed = packed ? h->transposed : 0;
    return GOL_OK;
}

static_assert(GOL_UNIT_FIELDS == 9 + kMaxNeighbours, "unit record layout");

int gol_plan_units(int64_t rows, int64_t words, int k, int tile_rows, int32_t *out, size_t cap, size_t *count) {
    if (rows < 1 || words < 1 || rows > INT32_MAX || words > INT32_MAX / 64 || !is_supported_k(k) || tile_rows < 1)
        return fail(GOL_EINVAL, "bad unit plan request");
    const UnitGrid g = unit_grid(rows, words, k, tile_rows);
    const size_t n = (size_t)g.nb * g.nt;
    if (n > (size_t)INT32_MAX) return fail(GOL_EINVAL, "unit plan of %zu units exceeds int32 unit ids", n);
    if (count) *count = n;
    if (!out) return GOL_OK;
    if (cap < n) return fail(GOL_EINVAL, "unit plan needs %zu records, buffer holds %zu", n, cap);
    std::vector<UnitDesc> us(n);
    fill_units(rows, words, 0, g, us.data(), 0);
    set_board_cost(us.data(), (int)n, k);
    for (size_t i = 0; i < n; ++i) {
        const UnitDesc &u = us[i];
        int32_t *o = out + i * GOL_UNIT_FIELDS;
        const int32_t f[8] = {u.r0, u.r_end, u.H, u.S, u.w0, u.U, u.mode, u.nnb};
        for (int j = 0; j < 8; ++j) o[j] = f[j];
        for (int j = 0; j < kMaxNeighbours; ++j) o[8 + j] = j < u.nnb ? u.nb[j] : -1;
        o[8 + kMaxNeighbours] = u.cost;
    }
    return GOL_OK;
}

int gol_kernel_launches(uint64_t *out) {
    if (!out) return fail(GOL_EINVAL, "null output");
    *out = launches_so_far();
    return GOL_OK;
}

int gol_device_info(int *sms, int64_t *l2, int *clk) {
    std::lock_guard<std::mutex> lk(g_mu);
    int rc = ensure_device();
    if (rc) return rc;
    if (sms) *sms = g_dev.sms;
    if (l2) *l2 = g_dev.l2;
    if (clk) *clk = g_dev.clock_khz;
    return GOL_OK;
}

int gol_probe_int_throughput(double *ops_per_s, double *seconds) {
    std::lock_guard<std::mutex> lk(g_mu);
    int rc = ensure_device();
    if (rc) return rc;
    const int block = 256, iters = 20000;
    const int grid = g_dev.sms * 8;
    Scratch sink((size_t)grid * 4);
    if (!sink.p) return fail(GOL_ENOMEM, "probe sink");
    cudaEvent_t a, b;
    CU(cudaEventCreate(&a));
    CU(cudaEventCreate(&b));
    CU(launch_int_probe((unsigned *)sink.p, 100, grid, block, g_stream));   // warm-up
    CU(cudaEventRecord(a, g_stream));
    CU(launch_int_probe((unsigned *)sink.p, iters, grid, block, g_stream));
    CU(cudaEventRecord(b, g_stream));
    CU(cudaEventSynchronize(b));
    float ms = 0;
    CU(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    const double ops = (double)grid * block * iters * int_probe_ops_per_iter();
    if (ops_per_s) *ops_per_s = ops / (ms * 1e-3);
    if (seconds) *seconds = ms * 1e-3;
    return GOL_OK;
}

int gol_debug_unfilled_wait(int64_t timeout_ms) {
    std::lock_guard<std::mutex> lk(g_mu);
    int rc = ensure_device();
    if (rc) return rc;
    if (timeout_ms < 1 || timeout_ms > 60000) return fail(GOL_EINVAL, "timeout out of range");
    Scratch ws(4096);
    if (!ws.p) return fail(GOL_ENOMEM, "debug workspace");
    PersistArgs a{};
    char *base = (char *)ws.p;
    a.boards = nullptr;
    a.units = nullptr;
    a.run = nullptr;
    a.next_pass = (int32_t *)(base + 0);
    a.join = (int32_t *)(base + 256);
    a.ctr = (int32_t *)(base + 512);
    a.qctr = (int32_t *)(base + 1024);
    a.ring = (int32_t *)(base + 2048);
    a.init_order = nullptr;
    a.sticky = g_dev.sticky;
    a.nunits = 0;        // no work ...
    a.total_tasks = 1;   // ... but one ticket: its slot is never filled
    a.hi_thr = INT64_MAX;
    a.hi_cap = 0;
    a.hi_init = 0;
    a.nwarps = kWarpsPerBlock;
    a.timeout_ns = timeout_ms * 1000000ll;
    CU(launch_sched_init(a, 0, g_stream));
    CU(launch_persistent<1>(a, true, 0, 1, g_stream));
    CU(cudaStreamSynchronize(g_stream));
    int32_t status = 0;
    CU(cudaMemcpy(&status, a.ctr + 3, sizeof status, cudaMemcpyDeviceToHost));
    int rc2 = take_sticky();
    if (status == GOL_ETIMEOUT && rc2 == GOL_ETIMEOUT) return GOL_ETIMEOUT;
    return fail(GOL_ECUDA, "bounded wait did not report a timeout (status %d, sticky %d)", status, rc2);
}

}  // extern "C"

// ===========================================================================
// Stepping a packed board without allocating device memory
// ===========================================================================
// Some callers cannot allocate device memory while they step a board: code
// running inside a memory pool or allocator of its own, code that must not
// synchronise with the device the way cudaMalloc/cudaFree may, or code that
// has a fixed memory budget reserved in advance.  This entry point takes the
// board and a spare buffer from the caller and keeps the scheduler's
// workspace (unit table, pass counters, work queue, status words) in one
// file-scope device array instead of allocating it.
namespace {
constexpr int kStaticMaxUnits = 4096;          // units of one board
constexpr int kStaticMaxTasks = 1 << 18;       // queue slots per launch
constexpr size_t kSaUnits = 256;               // offsets in the static workspace
constexpr size_t kSaInit = kSaUnits + sizeof(UnitDesc) * kStaticMaxUnits;
constexpr size_t kSaQctr = kSaInit + 4 * (size_t)kStaticMaxUnits;
constexpr size_t kSaRun = kSaQctr + 256;
static_assert(kSaQctr % 128 == 0 && kSaRun % 128 == 0, "queue counters and unit records are line aligned");
constexpr size_t kSaNext = kSaRun + sizeof(UnitRun) * kStaticMaxUnits;
constexpr size_t kSaJoin = kSaNext + 4 * (size_t)kStaticMaxUnits;
constexpr size_t kSaCtr = kSaJoin + 8 * (size_t)kStaticMaxUnits;
constexpr size_t kSaStatus = kSaCtr + 256;     // [0] status, [1] current buffer
constexpr size_t kSaRing = kSaStatus + 256;
constexpr size_t kStaticBytes = kSaRing + 4 * (size_t)kStaticMaxTasks;   // about 1.8 MiB

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) unsigned char g_static_workspace[kStaticBytes];

constexpr int kMaxDevices = 64;
char *g_static_base[kMaxDevices] = {};          // device address of the array, per device
UnitDesc g_static_units[kStaticMaxUnits];       // host copy of the unit table
int32_t g_static_init[kStaticMaxUnits];         // host copy of the units by queue ring
}  // namespace

extern "C" int gol_step_packed_noalloc(uint64_t *d_board, uint64_t *d_spare, int64_t rows, int64_t cols,
                                       int torus, int64_t generations, void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!d_board || !d_spare || d_board == d_spare) return fail(GOL_EINVAL, "need two distinct device buffers");
    if (rows < 1 || cols < 64 || cols % 64 != 0) return fail(GOL_EINVAL, "need rows >= 1 and cols a multiple of 64");
    if (rows > (int64_t(1) << 30)) return fail(GOL_EINVAL, "rows = %lld exceeds 2^30", (long long)rows);
    if (generations < 0) return fail(GOL_EINVAL, "negative generation count");
    const int64_t W = cols / 64;
    if ((W + kTileWords - 1) / kTileWords > kStaticMaxUnits)
        return fail(GOL_EINVAL, "cols = %lld exceeds the static workspace (at most %lld columns)", (long long)cols,
                    (long long)kTileWords * kStaticMaxUnits * 64);
    if (generations == 0) return GOL_OK;
    int dev = 0;
    CU(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(GOL_EINVAL, "device %d out of range", dev);
    if (!g_static_base[dev]) {   // first call on this device
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_workspace);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the static workspace");
        g_static_base[dev] = (char *)p;
    }
    char *base = g_static_base[dev];
    cudaStream_t s = (cudaStream_t)stream;
    int sms = 0;
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

    // plan: generations per pass and unit height as for gol_step, then taller
    // units until the board needs at most kStaticMaxUnits of them
    const TuneEntry te = tune_lookup(rows, cols);
    const int K = supported_k(std::max(1, te.k));
    int bps = 1;
    const int variant = plan_variant(K, 0);   // at most 4096 units: never the held-down variant
    CU(occupancy_for(K, torus != 0, variant, &bps));
    const int64_t slots = (int64_t)sms * std::max(1, bps) * kWarpsPerBlock;
    const int64_t npass_all = (generations + K - 1) / K;
    int h = std::max(1, te.rows);
    if (!g_opt_rows)
        h = capped_tile_rows(h, npass_all, K,
                             chain_fraction(1) * board_row_work(rows, W, npass_all) / (double)slots);
    UnitGrid g = unit_grid(rows, W, K, h);
    while (g.nb * g.nt > kStaticMaxUnits) {
        h = std::max(h + 1, (int)((int64_t)h * g.nb * g.nt / kStaticMaxUnits + 1));
        g = unit_grid(rows, W, K, h);
    }
    const int nunits = g.nb * g.nt;
    fill_units(rows, W, 0, g, g_static_units, 0);
    set_board_cost(g_static_units, nunits, K);

    CU(cudaMemcpyAsync(base + kSaUnits, g_static_units, sizeof(UnitDesc) * nunits, cudaMemcpyHostToDevice, s));
    CU(cudaMemsetAsync(base + kSaStatus, 0, 8, s));   // status and current-buffer words
    const int64_t nwords = rows * W;
    CU(launch_convert(d_board, d_board, nwords, true, s));

    PersistArgs a{};
    a.boards = (const BoardDesc *)base;
    a.units = (const UnitDesc *)(base + kSaUnits);
    a.init_order = (const int32_t *)(base + kSaInit);
    a.qctr = (int32_t *)(base + kSaQctr);
    a.run = (UnitRun *)(base + kSaRun);
    a.next_pass = (int32_t *)(base + kSaNext);
    a.join = (int32_t *)(base + kSaJoin);
    a.ctr = (int32_t *)(base + kSaCtr);
    a.ring = (int32_t *)(base + kSaRing);
    a.sticky = (int32_t *)(base + kSaStatus);
    a.nunits = nunits;
    a.timeout_ns = g_opt_timeout_ms * 1000000ll;
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)sms * std::max(1, bps), (nunits + kWarpsPerBlock - 1) / kWarpsPerBlock));
    a.nwarps = grid * kWarpsPerBlock;
    // launches of at most kStaticMaxTasks tasks each
    const int64_t passes_per_launch = std::max<int64_t>(1, kStaticMaxTasks / nunits);
    int cur = 0;
    for (int64_t left = generations; left > 0;) {
        const int64_t gens = std::min<int64_t>(left, passes_per_launch * K);
        BoardDesc bd{};
        bd.buf[0] = d_board;
        bd.buf[1] = d_spare;
        bd.cur = (int32_t *)(base + kSaStatus) + 1;
        bd.R = (int32_t)rows;
        bd.W = (int32_t)W;
        bd.gens = (int32_t)gens;
        bd.npass = (int32_t)((gens + K - 1) / K);
        bd.nunits = nunits;
        CU(cudaMemcpyAsync(base, &bd, sizeof bd, cudaMemcpyHostToDevice, s));
        a.total_tasks = nunits * bd.npass;
        plan_rings(g_static_units, nunits, 1, [&](int) { return bd.npass; }, a, g_static_init);
        CU(cudaMemcpyAsync(base + kSaInit, g_static_init, 4 * (size_t)nunits, cudaMemcpyHostToDevice, s));
        CU(launch_sched_init(a, 1, s));
        CU(launch_for(K, a, torus != 0, variant, grid, s));
        cur ^= bd.npass & 1;
        left -= gens;
    }
    // back to the interchange layout, into d_board
    CU(launch_convert(cur ? d_spare : d_board, d_board, nwords, false, s));
    CU(cudaStreamSynchronize(s));
    int32_t status = 0;
    CU(cudaMemcpy(&status, base + kSaStatus, sizeof status, cudaMemcpyDeviceToHost));
    if (status) return fail(status, "a device-side bounded wait gave up (status %d); the board is not valid", status);
    return GOL_OK;
}
