/*
 * gol.h -- C ABI of the GB300 Game of Life library (libgol.so).
 *
 * The operation is the generation step of Section 1 of "A performance
 * Analysis of the Game of Life based on parallel algorithm" (Ma, Chen,
 * Meng): every cell counts its eight horizontally, vertically and
 * diagonally adjacent neighbours and the four transitions of Section 1
 * are applied to all cells at once.  The board's left and right edges and
 * its top and bottom edges are adjacent (Section 2.2), i.e. the board is a
 * torus; a bounded board whose outside cells are dead is also offered
 * (torus = 0).
 *
 * Conventions shared by every call:
 *   - cells are uint8 0/1, row major, `rows` rows of `cols` columns;
 *   - the packed layout is uint64 words, row major, cols/64 words per row,
 *     bit j of word k of a row holding column 64*k + j;
 *   - host pointers belong to the caller and are not kept after the call
 *     returns; device state belongs to the handle;
 *   - every call returns GOL_OK (0) or a negative error code, and a
 *     message for the calling thread is available from gol_last_error();
 *   - stepping is asynchronous on the library's current CUDA stream
 *     (gol_set_stream); calls that return data to the host synchronise it.
 *     The tables a launch needs (unit plans, transfer plans) are copied to
 *     the device from page-locked staging blocks that the library keeps
 *     for the life of the process (at most 32, each reused once the copy
 *     from it has run), so queuing a launch does not wait for the work
 *     already on the stream.
 *
 * The library needs a CUDA GPU; there is no CPU path.  Calls made without
 * one return GOL_ECUDA.
 */
#ifndef GOL_H
#define GOL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GOL_OK 0
#define GOL_EINVAL (-1)   /* bad argument: null pointer, size mismatch, cell value not 0/1 ... */
#define GOL_ENOMEM (-2)   /* device allocation failed (including the allocator hook)          */
#define GOL_ECUDA (-3)    /* a CUDA call failed (no device, launch error ...)                  */
#define GOL_ETIMEOUT (-4) /* a bounded device-side wait gave up; the result is not valid       */
#define GOL_EBUSY (-5)    /* reserved; not returned: calls are serialised and stream-ordered      */

/* Board storage chosen at creation. */
#define GOL_LAYOUT_AUTO 0   /* packed, except a board with neither side a multiple of 64 whose     */
                            /* cells fit one thread-block cluster's shared memory: bytes           */
#define GOL_LAYOUT_PACKED 1 /* 64 cells per uint64, any rows, cols >= 1                            */
#define GOL_LAYOUT_BYTES 2  /* one uint8 per cell, any rows, cols >= 1                            */

typedef struct gol_board *gol_handle;

/* Creates a board of `rows` x `cols` dead cells (rows, cols >= 1) with the
 * wrap-around edges of Section 2.2 when torus != 0, dead outside otherwise.
 * Layout GOL_LAYOUT_AUTO.  Two device buffers of the board's size are
 * allocated (through the allocator hook if one is set).  Errors: GOL_EINVAL
 * for sizes < 1 or a null `out`, GOL_ENOMEM, GOL_ECUDA. */
int gol_create(int64_t rows, int64_t cols, int torus, gol_handle *out);

/* As gol_create with an explicit layout (GOL_LAYOUT_*).  Packed boards:
 *   - cols % 64 == 0: cols/64 words per row (stored transposed when that
 *     fills the warps better; the interchange layout is the same);
 *   - cols % 64 != 0, rows % 64 == 0: stored transposed (words along the
 *     height); it steps like any packed board, but has no packed word
 *     layout: gol_set_packed / gol_get_packed (and their device and batch
 *     forms) are GOL_EINVAL for it, gol_set / gol_get / gol_get_region work;
 *   - neither a multiple of 64: ceil(cols/64) words per row, the last one
 *     holding cols % 64 columns in its low bits (masked last word); its
 *     packed word layout has ceil(cols/64) words per row, padding bits are
 *     ignored on input and zero on output.  The step kernel carries the
 *     wrap across the partial word (a few more integer operations per word
 *     than a whole-word board). */
int gol_create_ex(int64_t rows, int64_t cols, int torus, int layout, gol_handle *out);

/* Releases the board.  The handle is invalid on return; the device memory
 * is freed once the work queued on the library's stream before this call
 * has finished (an event recorded here is polled by later calls, and
 * gol_set_allocator waits for all of them), so the call does not wait for
 * the device.  A null handle is GOL_EINVAL. */
int gol_destroy(gol_handle h);

/* Initial configuration (Section 1: "creating an initial configuration").
 * `cells` is host memory, rows*cols bytes, each 0 or 1; n must equal
 * rows*cols.  Any other value is GOL_EINVAL and leaves the board as it was.
 * Resets the generation counter to 0.  Synchronous. */
int gol_set(gol_handle h, const uint8_t *cells, size_t n);

/* Copies the current state to host `cells` (n == rows*cols bytes, 0/1).
 * Synchronises the stream first. */
int gol_get(gol_handle h, uint8_t *cells, size_t n);

/* Packed variants: `words` is host memory of nwords == rows*ceil(cols/64)
 * words in the packed layout.  Only for packed boards that have a word
 * layout (else GOL_EINVAL; see gol_create_ex).  gol_set_packed resets the
 * generation counter. */
int gol_set_packed(gol_handle h, const uint64_t *words, size_t nwords);
int gol_get_packed(gol_handle h, uint64_t *words, size_t nwords);

/* Device-to-device variants for callers that keep boards on the GPU:
 * `dwords` is device memory (nwords words, packed layout), read or written
 * on the library's current stream; asynchronous. */
int gol_set_packed_device(gol_handle h, const uint64_t *dwords, size_t nwords);
int gol_get_packed_device(gol_handle h, uint64_t *dwords, size_t nwords);

/* Many packed boards in one transfer.  `words` is host memory holding the
 * boards hs[0..n) one after the other, board i taking rows*cols/64 words in
 * the packed layout; nwords must equal the sum.  gol_set_packed_batch copies
 * the whole buffer to the device at once and scatters it into the boards
 * (handles must be distinct; generation counters reset to 0; asynchronous
 * when `words` is pinned).  gol_get_packed_batch gathers the boards'
 * current states into one device buffer, copies it to `words` and
 * synchronises.  When `words` is page-locked memory registered with CUDA
 * (cudaHostAlloc, cudaHostRegister) and no board of the transfer is stored
 * transposed, the scatter / gather kernel reads or
 * writes it in place, with no staging copy (GOL_OPT_ZERO_COPY = 0 turns
 * that off); otherwise the words go through a device staging buffer.
 * Non-packed boards are GOL_EINVAL. */
int gol_set_packed_batch(const gol_handle *hs, size_t n, const uint64_t *words, size_t nwords);
int gol_get_packed_batch(const gol_handle *hs, size_t n, uint64_t *words, size_t nwords);

/* As gol_get_packed_batch without waiting: the copy is queued on the
 * library's current stream and `words` holds the boards' states once that
 * work has run (wait on the stream, or an event recorded on it after this
 * call).  `words` must be page-locked memory for the call not to wait (a
 * pageable buffer makes the final device-to-host copy synchronous), and the
 * boards must not be stepped or destroyed on another stream meanwhile.
 * With it a caller keeps several batches in flight on several streams:
 * one batch's transfers overlap another's step. */
int gol_get_packed_batch_async(const gol_handle *hs, size_t n, uint64_t *words, size_t nwords);

/* Copies the nr x nc window whose top-left cell is (r0, c0) to host `out`
 * (nr*nc bytes, row major).  Window indices are taken modulo the board
 * size, so windows may straddle the wrap.  nr, nc >= 0. */
int gol_get_region(gol_handle h, int64_t r0, int64_t c0, int64_t nr, int64_t nc, uint8_t *out);

/* Allocation-free stepping of one packed torus or bounded board held by the
 * caller (the paper has no counterpart: this entry exists for callers that
 * cannot allocate device memory while they run, e.g. code inside its own
 * memory pool or with a fixed reserved budget).
 *   d_board  device memory, rows x cols/64 words in the packed layout; holds
 *            the initial state on entry and the state after `generations`
 *            steps on return;
 *   d_spare  device memory of the same size, distinct from d_board; its
 *            contents are overwritten;
 *   stream   the cudaStream_t to run on (null = default stream).
 * rows >= 1, cols a multiple of 64 and at most 30*4096*64 = 7864320,
 * generations >= 0.  The call allocates nothing: the scheduler's workspace
 * is a file-scope device array of about 1.8 MiB that every GPU loading the
 * library holds until the process exits.  The first call on a device looks
 * up that array's device address; make it before any stream capture.  All
 * calls share the array and it keeps the last call's contents (every call
 * re-initialises what must start at zero), so calls that overlapped on the
 * GPU would race: the library serialises its calls and each call waits for
 * its stream before returning.  Returns GOL_EINVAL for bad arguments or a
 * board too wide for the workspace, GOL_ETIMEOUT if a bounded device wait
 * gave up, GOL_ECUDA for CUDA errors.  GOL_EINVAL leaves both buffers
 * untouched; after GOL_ETIMEOUT or GOL_ECUDA the contents of d_board and
 * d_spare are unspecified (the board may be left in the library's internal
 * word order, or its live state in d_spare). */
int gol_step_packed_noalloc(uint64_t *d_board, uint64_t *d_spare, int64_t rows, int64_t cols, int torus,
                            int64_t generations, void *stream);

/* Advances the board by `generations` >= 0 steps (0 is a no-op).
 * Asynchronous; the result is bit-identical to applying the step of
 * Section 1 `generations` times.  Packed boards run several generations
 * per pass over the board (temporal blocking).  Returns GOL_ETIMEOUT if a
 * device-side wait gave up (the board is then in an unspecified state). */
int gol_step(gol_handle h, int64_t generations);

/* Advances handle hs[i] by generations[i] steps for i < n, all boards in
 * one persistent device launch (packed boards; byte boards are stepped
 * one by one).  Each board's result is bit-identical to gol_step on that
 * board alone.  Handles must be distinct (else GOL_EINVAL).  A repeated
 * call with the same handles and generation counts replays a captured CUDA
 * graph.  Asynchronous; errors as gol_step. */
int gol_step_batch(const gol_handle *hs, const int64_t *generations, size_t n);

/* Number of live cells (the quantity of the paper's Table 1).
 * Synchronous. */
int gol_population(gol_handle h, uint64_t *out);

/* Population trajectory (the form of the paper's Table 1, Section 3.1):
 * advances the board n times by `every` generations (every >= 1) and writes
 * the number of live cells after each advance to host out[0..n).  As
 * gol_population_trace_batch with one board.  Synchronous. */
int gol_population_trace(gol_handle h, int64_t every, size_t n, uint64_t *out);

/* Population trajectories of several boards at once: advances every board
 * hs[i] (distinct handles) by samples x every generations and writes its
 * number of live cells after each `every` generations to host
 * out[i * samples + k], k = 0 .. samples - 1.  Packed boards are stepped in
 * one persistent launch per torus flag (and per 2^24 generations), with
 * their passes aligned to the sampling period: at the end of each period
 * the step kernel adds up the live cells of the words it has just written.
 * Byte boards, and periods longer than 2^24 generations, are stepped and
 * counted sample by sample.  Synchronous.  GOL_EINVAL for null pointers,
 * every < 1, repeated or invalid handles. */
int gol_population_trace_batch(const gol_handle *hs, size_t n, int64_t every, size_t samples, uint64_t *out);

/* Generations applied since the last gol_set / gol_set_packed. */
int gol_generation(gol_handle h, int64_t *out);

/* Board geometry: rows, cols, torus flag and layout (GOL_LAYOUT_PACKED or
 * GOL_LAYOUT_BYTES). Any output pointer may be null. */
int gol_info(gol_handle h, int64_t *rows, int64_t *cols, int *torus, int *layout);

/* Waits for the library's current stream and reports any device-side
 * error recorded by earlier asynchronous calls on this handle. */
int gol_sync(gol_handle h);

/* Sets the CUDA stream (a cudaStream_t, e.g. a torch stream's handle) on
 * which subsequent calls of the calling process run; null selects the
 * default stream. */
int gol_set_stream(void *cuda_stream);

/* Routes device allocations through alloc(size, ctx) / free(ptr, ctx)
 * (e.g. the PyTorch caching allocator).  Passing two nulls restores
 * cudaMalloc / cudaFree.  Boards keep the allocator they were made with. */
int gol_set_allocator(void *(*alloc_fn)(size_t, void *), void (*free_fn)(void *, void *), void *ctx);

/* Message for the last error of the calling thread ("" if none). */
const char *gol_last_error(void);

/* Tuning knobs (process wide).  Keys:
 *   GOL_OPT_GENS_PER_PASS  generations per pass over a packed board (1, 2,
 *                          3, 4, 5, 6, 7, 8 or 16; 0 = let the autotune table
 *                          decide)
 *   GOL_OPT_TILE_ROWS      rows per warp strip of a packed board (>= 1;
 *                          0 = autotune table, shortened for boards with
 *                          many passes so that no chain of passes dominates)
 *   GOL_OPT_USE_GRAPHS     1 = capture/replay gol_step_batch in CUDA graphs
 *   GOL_OPT_WAIT_TIMEOUT_MS  limit of the device-side bounded waits
 *                          (default 5000 ms without progress)
 *   GOL_OPT_ORIENTATION    storage of packed boards created afterwards with
 *                          rows % 64 == 0: 0 = the library stores the board
 *                          transposed when that fills the warps better,
 *                          1 = never transposed, 2 = always transposed.  The
 *                          interchange layout and every result are the same.
 *   GOL_OPT_CHAIN_PERMILLE  planner bound on one board's chain of passes,
 *                          in thousandths of the average work per warp slot
 *                          (0 = 700 for one board, 500 for several); boards
 *                          above it get shorter units
 *   GOL_OPT_PIPELINE       0 = the step kernel shifts its three-row windows
 *                          by register moves (fewer registers, more warps),
 *                          1 = it rotates them by renaming (fewer issued
 *                          instructions), 2 = renaming with skewed stages
 *                          (stage g works one row behind stage g - 1, so the
 *                          stages of a row step are independent), 3 = 1 held
 *                          to three warps per scheduler at 8 generations per
 *                          pass, -1 (default) = 3 for 8 generations per pass
 *                          and many units per warp, else 1; results are
 *                          identical
 *   GOL_OPT_ZERO_COPY      1 (default): many-board transfers read and write
 *                          pinned host buffers in place; 0: always through a
 *                          device staging buffer and cudaMemcpyAsync
 *   GOL_OPT_CRITICAL_PERMILLE  a queued pass whose unit still has at least
 *                          this permille of the longest chain of passes ahead
 *                          of it is critical: idle warps take critical passes
 *                          first (0: one first-in first-out queue for all
 *                          passes; -1, the default: 750 when a launch steps
 *                          several boards, 0 for one board)
 *   GOL_OPT_BYTE_CLUSTER   1 (default): a byte board whose cells fit, one
 *                          bit each, in the shared memory of a thread-block
 *                          cluster of up to 8 CTAs (two buffers of
 *                          ceil(rows / n) rows of ceil(cols / 64) words per
 *                          CTA within 227 KiB) runs all its generations in
 *                          one launch of such a cluster (n: the smallest
 *                          that fits, doubled while a CTA would hold more
 *                          than 256 words); 2, 4, 8: that cluster size when
 *                          it fits; 0: one launch per generation (graph
 *                          replay when long)
 * Unknown keys or values are GOL_EINVAL. */
#define GOL_OPT_GENS_PER_PASS 1
#define GOL_OPT_TILE_ROWS 2
#define GOL_OPT_USE_GRAPHS 3
#define GOL_OPT_WAIT_TIMEOUT_MS 4
#define GOL_OPT_ORIENTATION 5
#define GOL_OPT_CHAIN_PERMILLE 6
#define GOL_OPT_PIPELINE 7
#define GOL_OPT_ZERO_COPY 8
#define GOL_OPT_BYTE_CLUSTER 9
#define GOL_OPT_CRITICAL_PERMILLE 10
int gol_set_option(int key, int64_t value);
int gol_get_option(int key, int64_t *value);

/* Autotune table: the (generations per pass, tile rows) pair used for
 * packed boards of a size class.  Size classes are keyed by
 * (ceil(log2(rows)), words per row class); gol_tune_set fixes the entry for
 * the class of (rows, cols), gol_tune_get reads the entry that would be
 * used. */
int gol_tune_set(int64_t rows, int64_t cols, int gens_per_pass, int tile_rows);
int gol_tune_get(int64_t rows, int64_t cols, int *gens_per_pass, int *tile_rows);
/* Removes every entry of the autotune table (built-in defaults apply). */
int gol_tune_reset(void);

/* The autotune table's class of a rows x cols board (host only):
 * *row_class = ceil(log2(rows)), *word_class = ceil(cols/64) when at most 32
 * words, else 32 + ceil(log2(words)).  Boards are looked up by their stored
 * shape (gol_board_storage), so a board stored transposed uses the class of
 * cols x rows. */
int gol_tune_class(int64_t rows, int64_t cols, int *row_class, int *word_class);

/* How a board is stored on the device (host only): *srows stored rows of
 * *swords words (packed boards; a byte board reports rows and 0 words),
 * *transposed = 1 when stored row c holds board column c.  Any output
 * pointer may be null. */
int gol_board_storage(gol_handle h, int64_t *srows, int64_t *swords, int *transposed);

/* Unit plan of a packed step (host only, no device needed).  Describes the
 * units a persistent launch uses for one board stored as `rows` x `words`
 * resident words per row (a board of cols % 64 == 0 is stored rows x
 * cols/64; one stored transposed is stored cols x rows/64), with
 * `gens_per_pass` generations per pass (a supported value, see
 * gol_tune_set) and `tile_rows` rows per unit (before any chain cap a batch
 * launch applies).  A unit is the rectangle of output cells one warp
 * produces per pass: the spatial blocking of Section 2.2 with the temporal
 * halo of K rows and one word.  *count receives the number of units; when
 * `out` is not NULL it must hold `cap` >= *count records of
 * GOL_UNIT_FIELDS int32 each:
 *   [0] r0, [1] r_end   output rows [r0, r_end) of the unit's row block
 *   [2] H               rows per segment
 *   [3] S               segments: full-row units split their row block into
 *                       S segments of H rows (the last one clipped), tiled
 *                       units have S = 1
 *   [4] w0, [5] U       output words [w0, w0 + U)
 *   [6] mode            0 = full rows (words <= 32), 1 = word tile
 *   [7] nnb             neighbour units (<= 8): those whose output the
 *                       unit's halo reads, which are also those that read
 *                       the unit's output
 *   [8 .. 15]           neighbour unit indices, -1 past nnb
 *   [16] cost           row iterations of a pass of the board's tallest
 *                       unit, H + 2K
 * Unit i covers row block i / nt and tile i % nt, where nt is the number of
 * tiles.  Returns GOL_EINVAL for bad arguments, a plan of more than
 * INT32_MAX units, or a short buffer. */
#define GOL_UNIT_FIELDS 17
int gol_plan_units(int64_t rows, int64_t words, int gens_per_pass, int tile_rows, int32_t *out, size_t cap,
                   size_t *count);

/* Number of kernels the library has launched in this process (host side
 * count: each launch adds one, each replay of a graph the library captured
 * adds the graph's kernels). */
int gol_kernel_launches(uint64_t *out);

/* Device facts used for rooflines: SM count, L2 bytes, SM clock (kHz). */
int gol_device_info(int *sm_count, int64_t *l2_bytes, int *sm_clock_khz);

/* Integer-pipe throughput probe: runs a kernel of independent 32-bit
 * LOP3/funnel-shift chains in the step's instruction mix on every SM and
 * returns operations per second in *ops_per_s and the kernel time. */
int gol_probe_int_throughput(double *ops_per_s, double *seconds);

/* Test hook for the bounded device-side waits: launches the batch
 * scheduler with one more work ticket than there is work, so that one
 * waiter waits for a slot that nothing fills; with a timeout of
 * `timeout_ms` it must give up and the call must return GOL_ETIMEOUT while
 * the context stays usable. */
int gol_debug_unfilled_wait(int64_t timeout_ms);

#ifdef __cplusplus
}
#endif

#endif /* GOL_H */
