// Internal declarations shared by the library's translation units.
//
// Packed boards: R rows of W uint64 words, row major, no padding; bit j of
// word k holds column 64k + j.  Each board owns two such buffers and a
// device int `cur` naming the one that holds the current generation.
//
// Device-resident word layout.  The interchange layout (bit j of word k =
// column 64k + j) is converted on every upload and download to the
// resident layout, in which the low 32 bits of a word hold the word's even
// columns (bit j = column 64k + 2j) and the high 32 bits its odd columns
// (bit 32 + j = column 64k + 2j + 1).  With that split the east neighbour of
// an even column and the west neighbour of an odd column sit at the same bit
// of the other half, so a row's horizontal neighbour planes take 2 funnel
// shifts per word instead of 4.
//
// A packed step is organised in "units": the rectangle of output cells one
// warp produces per pass.  A pass advances a unit by kk <= K generations,
// reading the previous pass's buffer (with a K-row and one-word halo) and
// writing the other buffer.  Passes of neighbouring units are ordered by
// the dataflow scheduler in wavefront.cuh.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gol.h"

namespace gol {

constexpr int kMaxNeighbours = 8;   // units whose output a unit's halo can touch
constexpr int kTileWords = 30;      // output words of a tiled warp (32 lanes - 2 halo lanes)
constexpr int kWarpsPerBlock = 2;   // persistent kernel: 64-thread blocks (fine occupancy steps)

enum UnitMode : int32_t { kUnitFull = 0, kUnitTiled = 1 };

// One board in a launch (device memory).
struct BoardDesc {
    uint64_t *buf[2];
    int32_t *cur;     // device: index of the buffer holding the current state
    int32_t R;        // rows
    int32_t W;        // words per row
    int32_t npass;    // passes in this launch (>= 1)
    int32_t gens;     // generations in this launch (>= npass)
    int32_t nunits;   // units of this board
    int32_t ppp;      // population trace: passes per sampling period (0 = no trace); see pass_gens
    int32_t pop_off;  // population trace: the board's first sample slot in PersistArgs::pop
    int32_t last_bits;// masked last word: valid columns of each row's last word (1..63), 0 = all 64
};

// One unit (device memory).
//  kUnitFull : W <= 32, a row fits one warp; lanes are S segments of W
//              lanes, segment s produces rows [r0 + s*H, r0 + (s+1)*H)
//              clipped to r_end; horizontal wrap happens inside the segment.
//  kUnitTiled: W > 32; lane l holds word (w0 - 1 + l) mod W for l < U + 2,
//              lanes 1..U produce words w0 .. w0+U-1 of rows [r0, r_end).
struct UnitDesc {
    int32_t board;
    int32_t r0, r_end;
    int32_t H;        // segment height
    int32_t S;        // segments (kUnitFull) or 1
    int32_t w0, U;    // kUnitTiled word range; kUnitFull: 0, W
    int32_t mode;
    int32_t nnb;      // neighbour units (same board), whose passes bound this one's
    int32_t nb[kMaxNeighbours];
    int32_t cost;     // row iterations of a pass of the board's tallest unit (H + 2K), the same
                      // for all units of a board: a pass's share of the rest of its chain
};

// What a warp needs to run a pass of one unit, in one 128-byte record:
// the unit's geometry, its board's fields and the board's current buffer at
// the start of the launch (a board's `cur` only changes after all its units
// have run their last pass).  Written by sched_init_kernel at the start of
// every launch from the unit and board tables.
struct __align__(128) UnitRun {
    uint64_t *buf[2];
    int32_t *curp;     // the board's device `cur`
    int32_t board, R, W, npass, gens, nunits, cur;
    int32_t r0, r_end, H, S, w0, U, mode, nnb;
    int32_t nb[kMaxNeighbours];
    int32_t cost;      // UnitDesc::cost
    int32_t ppp;       // BoardDesc::ppp
    int32_t pop_off;   // BoardDesc::pop_off
};
static_assert(sizeof(UnitRun) == 128, "UnitRun is one 128-byte line");

// Kernel arguments of the persistent dataflow kernel.
struct PersistArgs {
    const BoardDesc *boards;
    const UnitDesc *units;
    UnitRun *run;       // [nunits] per-launch unit records (sched_init_kernel)
    int32_t *next_pass; // [nunits] the pass a queued unit runs next (set when it is claimed)
    int32_t *join;      // [2 * nunits] join counters, one per pass parity
    int32_t *ring;      // [total_tasks] work queues, -1 = empty slot: the critical ring
                        // [0, hi_cap), then the other ring [hi_cap, total_tasks)
    int32_t *qctr;      // 128-byte line: [0] critical head, [1] critical tail,
                        // [2] other ring's tickets, [3] other ring's tail
    int32_t *ctr;       // [2] tasks completed, [3] status,
                        // [4 + b] units of board b that finished all passes
    int32_t *sticky;    // process-wide error word read by synchronising calls
    int32_t nunits;
    int32_t total_tasks;
    int64_t timeout_ns; // bounded waits give up after this long without progress
    int64_t hi_thr;     // a pass is critical when (npass - pass + 1) * cost >= hi_thr
    int32_t hi_cap;     // critical passes of the launch (the critical ring's size)
    int32_t hi_init;    // first passes in the critical ring at launch (units 0 .. hi_init - 1
                        // of init_order), the rest in the other ring
    int32_t nwarps;     // warps of the launch; warp w < hi_init starts with critical slot w
    int32_t pad;
    const int32_t *init_order;   // [nunits] units by ring: critical first passes, then the others
    unsigned long long *pop;     // population trace: live cells per (board, sample) slot, or null
};

// One board of a many-board transfer: `nwords` words of the board buffer
// `board` live at word `offset` of a contiguous staging buffer.
__host__ __device__ __forceinline__ uint64_t compress_even_bits(uint64_t v) {
    v &= 0x5555555555555555ull;
    v = (v | (v >> 1)) & 0x3333333333333333ull;
    v = (v | (v >> 2)) & 0x0F0F0F0F0F0F0F0Full;
    v = (v | (v >> 4)) & 0x00FF00FF00FF00FFull;
    v = (v | (v >> 8)) & 0x0000FFFF0000FFFFull;
    return (v | (v >> 16)) & 0x00000000FFFFFFFFull;
}
__host__ __device__ __forceinline__ uint64_t spread_to_even_bits(uint64_t v) {
    v &= 0x00000000FFFFFFFFull;
    v = (v | (v << 16)) & 0x0000FFFF0000FFFFull;
    v = (v | (v << 8)) & 0x00FF00FF00FF00FFull;
    v = (v | (v << 4)) & 0x0F0F0F0F0F0F0F0Full;
    v = (v | (v << 2)) & 0x3333333333333333ull;
    return (v | (v << 1)) & 0x5555555555555555ull;
}
// interchange layout -> resident layout
__host__ __device__ __forceinline__ uint64_t to_resident(uint64_t w) {
    return compress_even_bits(w) | (compress_even_bits(w >> 1) << 32);
}
// resident layout -> interchange layout
__host__ __device__ __forceinline__ uint64_t to_interchange(uint64_t w) {
    return spread_to_even_bits(w) | (spread_to_even_bits(w >> 32) << 1);
}
// bit of column c (0 <= c < 64) of a resident word
__host__ __device__ __forceinline__ int resident_bit(int c) { return (c & 1) ? 32 + (c >> 1) : (c >> 1); }

struct CopyDesc {
    uint64_t *buf[2];   // the board's buffers: scatter writes buf[0], gather reads buf[*cur]
    int32_t *cur;       // the board's device `cur` (scatter resets it to 0)
    int64_t offset;
    int64_t nwords;
    int64_t rows;       // board geometry in the interchange layout
    int64_t words;
    int32_t transposed; // board stored transposed (see gol_api.cu)
    int32_t last_bits;  // masked last word: valid columns of the last word of a row, 0 = all 64
    int64_t block0;     // first block of this board in the copy grid
};

// Copy grid: a board takes ceil(words / kCopyWordsPerBlock) blocks, or, when
// stored transposed, one block per super-tile of kSuper x kSuper tiles of
// 64 x 64 cells; at least one; the boards' blocks are consecutive.
constexpr int64_t kCopyWordsPerBlock = 4096;
constexpr int kSuper = 8;
__host__ __device__ __forceinline__ int64_t copy_blocks(const CopyDesc &c) {
    if (c.transposed) {
        const int64_t n = ((c.rows / 64 + kSuper - 1) / kSuper) * ((c.words + kSuper - 1) / kSuper);
        return n > 0 ? n : 1;
    }
    return c.nwords > 0 ? (c.nwords + kCopyWordsPerBlock - 1) / kCopyWordsPerBlock : 1;
}

// Launchers (one translation unit per K).  Return cudaGetLastError().
// variant 0: window rows shift by register moves (fewer registers);
// variant 1: window slots rotate by renaming (fewer issued instructions).
template <int K>
cudaError_t launch_persistent(const PersistArgs &a, bool torus, int variant, int grid, cudaStream_t s);
template <int K>
cudaError_t persistent_occupancy(bool torus, int variant, int *blocks_per_sm);

// Kernel launch count of the process (kernels_util.cu): every launcher adds
// the kernels it launches; launches recorded into a CUDA graph while the
// library captures one are not counted (set_capturing), each replay of such
// a graph adds the graph's kernel count instead.
void count_launches(int n);
void set_capturing(bool on);
uint64_t launches_so_far();

// Utility kernels (kernels_util.cu).
cudaError_t launch_sched_init(const PersistArgs &a, int nboards, cudaStream_t s);
cudaError_t launch_byte_step(const uint8_t *in, uint8_t *out, int64_t R, int64_t C, int torus,
                             cudaStream_t s);
cudaError_t launch_pack(const uint8_t *cells, uint64_t *words, int64_t R, int64_t W, int32_t *bad,
                        cudaStream_t s);
cudaError_t launch_check_bytes(const uint8_t *cells, int64_t n, int32_t *bad, cudaStream_t s);
cudaError_t launch_unpack(const uint64_t *words, uint8_t *cells, int64_t R, int64_t W, cudaStream_t s);
cudaError_t launch_region_packed(const uint64_t *words, int64_t R, int64_t C, int64_t r0, int64_t c0, int64_t nr,
                                 int64_t nc, uint8_t *out, bool transposed, cudaStream_t s);
// boards of any width stored transposed (R % 64 == 0), to / from one byte per cell
cudaError_t launch_pack_transposed(const uint8_t *cells, int64_t R, int64_t C, uint64_t *store, int32_t *bad,
                                   cudaStream_t s);
cudaError_t launch_unpack_transposed(const uint64_t *store, int64_t R, int64_t C, uint8_t *cells, cudaStream_t s);
// R x W interchange words <-> resident storage (the transpose when
// `transposed`); to_res selects the direction.  src and dst must differ when
// transposed.
cudaError_t launch_orient(const uint64_t *src, uint64_t *dst, int64_t R, int64_t W, bool transposed, bool to_res,
                          cudaStream_t s, int last_bits = 0);
// rows of any width C (W = ceil(C / 64) words per row, padding bits zero) to / from one byte per cell
cudaError_t launch_pack_rows(const uint8_t *cells, uint64_t *words, int64_t R, int64_t C, int32_t *bad,
                             cudaStream_t s);
cudaError_t launch_unpack_rows(const uint64_t *words, uint8_t *cells, int64_t R, int64_t C, cudaStream_t s);
cudaError_t launch_region_bytes(const uint8_t *cells, int64_t R, int64_t C, int64_t r0, int64_t c0,
                                int64_t nr, int64_t nc, uint8_t *out, cudaStream_t s);
cudaError_t launch_popcount_packed(const uint64_t *words, int64_t n, unsigned long long *out,
                                   cudaStream_t s);
cudaError_t launch_popcount_bytes(const uint8_t *cells, int64_t n, unsigned long long *out,
                                  cudaStream_t s);
// Byte boards resident, one bit per cell, in one thread-block cluster
// (kernels_util.cu): the cluster size for an R x C board (the smallest power
// of two whose CTAs hold two buffers of their strip), 0 when none does.
constexpr int kByteClusterMax = 8;                 // CTAs per cluster (portable size)
constexpr int64_t kByteClusterBytes = 227 * 1024;  // shared memory per CTA
int byte_cluster_size(int64_t R, int64_t C);
constexpr int64_t kByteWordsPerCta = 256;          // auto cluster size: words per CTA at most (if it can)
int byte_cluster_choice(int64_t R, int64_t C, int want);
cudaError_t launch_byte_cluster(const uint8_t *in, uint8_t *out, int64_t R, int64_t C, int torus, int G, int want,
                                cudaStream_t s);
cudaError_t launch_convert(const uint64_t *src, uint64_t *dst, int64_t n, bool to_res, cudaStream_t s);
cudaError_t launch_scatter_boards(const CopyDesc *d, const int32_t *block_board, int64_t blocks, const uint64_t *staging,
                                  cudaStream_t s);
cudaError_t launch_gather_boards(const CopyDesc *d, const int32_t *block_board, int64_t blocks, uint64_t *staging,
                                 cudaStream_t s);
cudaError_t launch_int_probe(unsigned *sink, int iters, int grid, int block, cudaStream_t s);
int int_probe_ops_per_iter();   // 32-bit integer operations per thread per probe iteration

}  // namespace gol
