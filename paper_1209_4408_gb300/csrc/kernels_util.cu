// Byte-per-cell step, layout conversion, population count, scheduler
// initialisation and the integer-throughput probe.
#include <atomic>
#include <cooperative_groups.h>

#include "gol_internal.h"
#include "wavefront.cuh"

namespace gol {

namespace {

constexpr int kBlock = 256;

int grid_for(int64_t n, int block = kBlock, int64_t cap = 1 << 20) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// --- scheduler state ------------------------------------------------------
__global__ void sched_init_kernel(PersistArgs a, int nboards) {
    const int64_t n = max(max((int64_t)a.nunits, (int64_t)a.total_tasks), (int64_t)max(nboards, 32));
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < a.nunits) {
            const UnitDesc u = a.units[i];
            const BoardDesc b = a.boards[u.board];
            UnitRun r;
            r.buf[0] = b.buf[0];
            r.buf[1] = b.buf[1];
            r.curp = b.cur;
            r.board = u.board;
            r.R = b.R;
            r.W = b.W;
            r.npass = b.npass;
            r.gens = b.gens;
            r.nunits = b.nunits;
            r.cur = *b.cur;
            r.r0 = u.r0;
            r.r_end = u.r_end;
            r.H = u.H;
            r.S = u.S;
            r.w0 = u.w0;
            r.U = u.U;
            r.mode = u.mode | (b.last_bits << 8);   // the kernel reads the masked width from bits 8..15
            r.nnb = u.nnb;
            for (int k = 0; k < kMaxNeighbours; ++k) r.nb[k] = u.nb[k];
            r.cost = u.cost;
            r.ppp = b.ppp;
            r.pop_off = b.pop_off;
            a.run[i] = r;
            a.next_pass[i] = 1;            // every unit's first pass is queued below
            a.join[2 * i] = u.nnb + 1;     // join counters of both pass parities count down
            a.join[2 * i + 1] = u.nnb + 1; // the completions a pass waits for
        }
        if (i < a.total_tasks) {
            // critical ring: its first hi_init slots; other ring: its first nunits - hi_init
            int32_t v = -1;
            if (i < a.hi_cap) {
                if (i < a.hi_init) v = a.init_order[i];
            } else if (i - a.hi_cap < a.nunits - a.hi_init) {
                v = a.init_order[a.hi_init + (i - a.hi_cap)];
            }
            a.ring[i] = v;
        }
        if (i < nboards) a.ctr[4 + i] = 0;
        if (i < 32) {
            int32_t v = 0;
            if (i == 0) v = min(a.hi_init, a.nwarps);    // critical tickets: past the passes dealt at launch
            if (i == 1) v = a.hi_init;
            if (i == 3) v = a.nunits - a.hi_init;
            a.qctr[i] = v;
        }
        if (i == 0) {
            a.ctr[0] = 0;
            a.ctr[1] = 0;
            a.ctr[2] = 0;         // tasks completed
            a.ctr[3] = 0;         // status
        }
    }
}

// --- byte-per-cell step (Section 1, one uint8 per cell) -------------------
__global__ void byte_step_kernel(const uint8_t *__restrict__ in, uint8_t *__restrict__ out,
                                 int64_t R, int64_t C, int torus) {
    const int64_t n = R * C;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / C, c = i - r * C;
        int cnt = 0;
#pragma unroll
        for (int dr = -1; dr <= 1; ++dr) {
            int64_t rr = r + dr;
            bool rin = true;
            if (rr < 0) {
                rr = R - 1;
                rin = torus;
            } else if (rr >= R) {
                rr = 0;
                rin = torus;
            }
#pragma unroll
            for (int dc = -1; dc <= 1; ++dc) {
                if (dr == 0 && dc == 0) continue;
                int64_t cc = c + dc;
                bool cin = true;
                if (cc < 0) {
                    cc = C - 1;
                    cin = torus;
                } else if (cc >= C) {
                    cc = 0;
                    cin = torus;
                }
                if (rin && cin) cnt += in[rr * C + cc] != 0;
            }
        }
        const bool alive = in[i] != 0;
        out[i] = (cnt == 3) || (alive && cnt == 2);
    }
}

// --- layout conversion ------------------------------------------------------
// four 0/1 bytes of a little-endian uint32 -> 4 bits
__device__ __forceinline__ uint32_t gather4(uint32_t x) {
    return (x | (x >> 7) | (x >> 14) | (x >> 21)) & 0xFu;
}
__device__ __forceinline__ uint32_t spread4(uint32_t b) {
    return (b & 1u) | ((b & 2u) << 7) | ((b & 4u) << 14) | ((b & 8u) << 21);
}

__global__ void pack_kernel(const uint8_t *__restrict__ cells, uint64_t *__restrict__ words,
                            int64_t nwords, int32_t *bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nwords;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 *p = reinterpret_cast<const uint4 *>(cells + i * 64);
        uint64_t w = 0;
        uint32_t any_high = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 v = p[q];
            const uint32_t parts[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                any_high |= parts[e] & 0xFEFEFEFEu;
                w |= (uint64_t)gather4(parts[e]) << (16 * q + 4 * e);
            }
        }
        if (any_high) atomicExch(bad, 1);
        words[i] = w;
    }
}

__global__ void check_bytes_kernel(const uint8_t *__restrict__ cells, int64_t n, int32_t *bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (cells[i] > 1) atomicExch(bad, 1);
}

__global__ void unpack_kernel(const uint64_t *__restrict__ words, uint8_t *__restrict__ cells,
                              int64_t nwords) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nwords;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t w = words[i];
        uint4 *p = reinterpret_cast<uint4 *>(cells + i * 64);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint4 v;
            v.x = spread4((uint32_t)(w >> (16 * q + 0)) & 0xFu);
            v.y = spread4((uint32_t)(w >> (16 * q + 4)) & 0xFu);
            v.z = spread4((uint32_t)(w >> (16 * q + 8)) & 0xFu);
            v.w = spread4((uint32_t)(w >> (16 * q + 12)) & 0xFu);
            p[q] = v;
        }
    }
}

__device__ __forceinline__ int64_t wrap(int64_t x, int64_t m) {
    int64_t r = x % m;
    return r < 0 ? r + m : r;
}

__global__ void region_packed_kernel(const uint64_t *__restrict__ words, int64_t R, int64_t C,
                                     int64_t r0, int64_t c0, int64_t nr, int64_t nc,
                                     uint8_t *__restrict__ out, bool transposed) {
    const int64_t n = nr * nc, W = (C + 63) / 64;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t y = i / nc, x = i - y * nc;
        const int64_t r = wrap(r0 + y, R), c = wrap(c0 + x, C);
        // transposed storage holds cell (r, c) at stored row c, stored column r
        const int64_t sr = transposed ? c : r, sc = transposed ? r : c;
        const int64_t sw = transposed ? R / 64 : W;
        out[i] = (uint8_t)((words[sr * sw + (sc >> 6)] >> resident_bit((int)(sc & 63))) & 1u);
    }
}

__global__ void region_bytes_kernel(const uint8_t *__restrict__ cells, int64_t R, int64_t C,
                                    int64_t r0, int64_t c0, int64_t nr, int64_t nc,
                                    uint8_t *__restrict__ out) {
    const int64_t n = nr * nc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t y = i / nc, x = i - y * nc;
        out[i] = cells[wrap(r0 + y, R) * C + wrap(c0 + x, C)];
    }
}

template <typename T>
__global__ void popcount_kernel(const T *__restrict__ v, int64_t n, unsigned long long *out) {
    unsigned long long s = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (sizeof(T) == 8)
            s += __popcll((unsigned long long)v[i]);
        else
            s += v[i] != 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

// --- byte-per-cell boards resident in one thread-block cluster -----------------
// A byte board whose cells fit, one bit each, in the shared memory of a
// cluster of n <= kByteClusterMax CTAs runs G generations in one launch.
// CTA k packs rows [R k / n, R (k + 1) / n) into words (bit j of word w =
// column 64 w + j, W = ceil(C / 64) words per row, the last one holding
// C - 64 (W - 1) columns), double-buffered, steps them with the same
// bit-sliced rule as the packed boards, and unpacks the result.  The rows just
// above and below a strip are read from the neighbouring CTAs' shared memory
// (distributed shared memory; wrapping across the cluster on the torus, zero
// otherwise) and a cluster barrier separates generations.  Every strip has at
// least one row (n <= R), and the horizontal wrap takes column C - 1 / 0 from
// wherever it sits, so tiny tori alias exactly as the per-cell kernel does.
__device__ __forceinline__ uint64_t byte_rule(uint64_t t0, uint64_t t1, uint64_t m0, uint64_t m1, uint64_t b0,
                                              uint64_t b1, uint64_t a) {
    // S = (t0 + m0 + b0) + 2 (t1 + m1 + b1) = u0 + 2 (u1 + p) + 4 q; next = S==3 | (a & S==4)
    const uint64_t u0 = t0 ^ m0 ^ b0, u1 = (t0 & m0) | (b0 & (t0 ^ m0));
    const uint64_t p = t1 ^ m1 ^ b1, q = (t1 & m1) | (b1 & (t1 ^ m1));
    const uint64_t e = p ^ u1;
    return (u0 & e & ~q) | (~u0 & ~e & (p ^ q) & a);
}

// Row-sum planes (s0 + 2 s1 = west + cell + east) of word w of a row.
__device__ __forceinline__ void byte_row_sum(const uint64_t *row, int w, int W, int last_bits, bool torus,
                                             uint64_t &s0, uint64_t &s1) {
    const uint64_t x = row[w];
    uint64_t wc, ec;   // west neighbour of bit 0, east neighbour of the top valid bit
    if (w > 0) wc = row[w - 1] >> 63;
    else wc = torus ? (row[W - 1] >> (last_bits - 1)) & 1 : 0;
    if (w < W - 1) ec = row[w + 1] & 1;
    else ec = torus ? row[0] & 1 : 0;
    const uint64_t west = (x << 1) | wc;
    const uint64_t east = w < W - 1 ? (x >> 1) | (ec << 63) : (x >> 1) | (ec << (last_bits - 1));
    s0 = west ^ x ^ east;
    s1 = (west & x) | (east & (west ^ x));
}

// CLUSTERED: n > 1 CTAs exchanging halo rows through distributed shared
// memory; otherwise one CTA whose strip is the whole board.
template <bool CLUSTERED>
__global__ void byte_resident_kernel(const uint8_t *__restrict__ in, uint8_t *__restrict__ out, int R, int C,
                                     int torus, int G) {
    extern __shared__ uint64_t smw[];
    namespace cg = cooperative_groups;
    const int n = CLUSTERED ? (int)cg::this_cluster().num_blocks() : 1;
    const int k = CLUSTERED ? (int)cg::this_cluster().block_rank() : 0;
    const int W = (C + 63) / 64, last_bits = C - 64 * (W - 1);
    const uint64_t last_mask = last_bits == 64 ? ~0ull : (1ull << last_bits) - 1;
    const int hmax = (R + n - 1) / n;
    const int r0 = (int)((int64_t)R * k / n), h = (int)((int64_t)R * (k + 1) / n) - r0;
    const int up = (k + n - 1) % n, dn = (k + 1) % n;
    const int h_up = (int)((int64_t)R * (up + 1) / n - (int64_t)R * up / n);
    const bool has_up = torus || k > 0, has_dn = torus || k < n - 1;
    const size_t buf_words = (size_t)hmax * W;
    const int nw = h * W;
    // this thread's first word (row lr0, word w0) and the stride in rows / words
    const int lr0 = (int)threadIdx.x / W, w0 = (int)threadIdx.x - lr0 * W;
    const int step_r = (int)blockDim.x / W, step_w = (int)blockDim.x - step_r * W;
    for (int i = threadIdx.x, lr = lr0, w = w0; i < nw; i += blockDim.x) {
        const uint8_t *src = in + (int64_t)(r0 + lr) * C + 64 * w;
        const int nb = w < W - 1 ? 64 : last_bits;
        uint64_t v = 0;
        for (int j = 0; j < nb; ++j) v |= (uint64_t)(src[j] != 0) << j;
        smw[i] = v;
        lr += step_r;
        w += step_w;
        if (w >= W) { w -= W; ++lr; }
    }
    if (CLUSTERED) cg::this_cluster().sync(); else __syncthreads();
    for (int g = 0; g < G; ++g) {
        const int cb = g & 1;
        const uint64_t *cur = smw + cb * buf_words;
        uint64_t *nxt = smw + (cb ^ 1) * buf_words;
        const uint64_t *above, *below;
        if (CLUSTERED) {
            above = cg::this_cluster().map_shared_rank(smw, up) + cb * buf_words + (size_t)(h_up - 1) * W;
            below = cg::this_cluster().map_shared_rank(smw, dn) + cb * buf_words;
        } else {
            above = cur + (size_t)(h - 1) * W;     // the torus wraps within the board
            below = cur;
        }
        for (int i = threadIdx.x, lr = lr0, w = w0; i < nw; i += blockDim.x) {
            const uint64_t *rm = cur + (size_t)lr * W;
            const uint64_t *ra = lr > 0 ? rm - W : (has_up ? above : nullptr);
            const uint64_t *rb = lr < h - 1 ? rm + W : (has_dn ? below : nullptr);
            uint64_t t0 = 0, t1 = 0, m0, m1, b0 = 0, b1 = 0;
            if (ra) byte_row_sum(ra, w, W, last_bits, torus, t0, t1);
            byte_row_sum(rm, w, W, last_bits, torus, m0, m1);
            if (rb) byte_row_sum(rb, w, W, last_bits, torus, b0, b1);
            uint64_t v = byte_rule(t0, t1, m0, m1, b0, b1, rm[w]);
            if (w == W - 1) v &= last_mask;
            nxt[i] = v;
            lr += step_r;
            w += step_w;
            if (w >= W) { w -= W; ++lr; }
        }
        if (CLUSTERED) cg::this_cluster().sync(); else __syncthreads();
    }
    const uint64_t *res = smw + (G & 1) * buf_words;
    for (int i = threadIdx.x; i < h * C; i += blockDim.x) {
        const int lr = i / C, c = i - lr * C;
        out[(int64_t)(r0 + lr) * C + c] = (uint8_t)((res[(size_t)lr * W + (c >> 6)] >> (c & 63)) & 1);
    }
}

// --- boards stored transposed straight from / to one byte per cell -----------
// Stored row j holds column j of the R x C board, word i of it rows
// [64 i, 64 i + 64) (resident layout); R % 64 == 0, C arbitrary.  Neighbouring
// threads take neighbouring columns, so each of the 64 byte rows a word
// gathers is read (or written) coalesced.  Bytes other than 0 / 1 set *bad.
__global__ void pack_transposed_kernel(const uint8_t *__restrict__ cells, int64_t R, int64_t C,
                                       uint64_t *__restrict__ store, int32_t *bad) {
    const int64_t sw = R / 64, n = sw * C;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / C, j = idx - i * C;
        const uint8_t *col = cells + 64 * i * C + j;
        uint64_t w = 0;
        bool b = false;
        for (int k = 0; k < 64; ++k) {
            const uint8_t v = col[(int64_t)k * C];
            b |= v > 1;
            w |= (uint64_t)(v & 1u) << k;
        }
        if (b) atomicExch(bad, 1);
        store[j * sw + i] = to_resident(w);
    }
}

__global__ void unpack_transposed_kernel(const uint64_t *__restrict__ store, int64_t R, int64_t C,
                                         uint8_t *__restrict__ cells) {
    const int64_t sw = R / 64, n = sw * C;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / C, j = idx - i * C;
        const uint64_t w = to_interchange(store[j * sw + i]);
        uint8_t *col = cells + 64 * i * C + j;
        for (int k = 0; k < 64; ++k) col[(int64_t)k * C] = (uint8_t)((w >> k) & 1u);
    }
}

// --- interchange <-> resident word layout ---------------------------------------
__global__ void convert_kernel(const uint64_t *src, uint64_t *dst, int64_t n, bool to_res) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t w = src[i];
        dst[i] = to_res ? to_resident(w) : to_interchange(w);
    }
}

// A warp transposes a 64 x 64 bit matrix held as lane l: a = row l,
// b = row l + 32 (bit j of a row = column j); afterwards lane l holds rows l
// and l + 32 of the transpose.  Six rounds of masked block swaps (32-row
// blocks within a lane, then 16, 8, 4, 2, 1 between lanes l and l ^ j).
__device__ __forceinline__ void transpose64_lanes(uint64_t &a, uint64_t &b) {
    const int lane = threadIdx.x & 31;
    uint64_t m = 0x00000000FFFFFFFFull;
    const uint64_t t = ((a >> 32) ^ b) & m;
    a ^= t << 32;
    b ^= t;
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        m ^= m << j;
        const uint64_t pa = __shfl_xor_sync(0xffffffffu, a, j), pb = __shfl_xor_sync(0xffffffffu, b, j);
        if (lane & j) {
            a ^= ((pa >> j) ^ a) & m;
            b ^= ((pb >> j) ^ b) & m;
        } else {
            a ^= (((a >> j) ^ pa) & m) << j;
            b ^= (((b >> j) ^ pb) & m) << j;
        }
    }
}

// One block of 256 threads (8 warps) moves a super-tile of kSuper x kSuper
// such tiles with full 64-byte rows on both sides.  src holds src_rows x
// src_w words (src_rows % 64 == 0); dst is its transpose, (64 src_w) x
// (src_rows / 64) words.  Super-tile (si, sj) covers tile rows
// ti in [8 si, 8 si + 8) and tile columns tj in [8 sj, 8 sj + 8): warp w
// reads rows 64 (8 si + w) + lane and + 32, words 8 sj .. 8 sj + 7 of each,
// transposes its tiles (transpose64_lanes) into shared memory, and the block then
// writes output rows 64 tj + r, words 8 si .. 8 si + 7.  Tiles past the
// edges of the board are skipped.  Every thread of the block must call it.
__device__ void transpose_super(const uint64_t *__restrict__ src, int64_t src_rows, int64_t src_w,
                                uint64_t *__restrict__ dst, int64_t si, int64_t sj, bool from_res, bool to_res) {
    __shared__ uint64_t sm[kSuper][64][kSuper + 1];   // [tile column][row][tile row], padded
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nti = src_rows / 64;
    const int nk = (int)min((int64_t)kSuper, src_w - kSuper * sj);   // tile columns present
    const int nw = (int)min((int64_t)kSuper, nti - kSuper * si);     // tile rows present
    if (w < nw) {
        const uint64_t *ra = src + (64 * (kSuper * si + w) + lane) * src_w + kSuper * sj;
        const uint64_t *rb = ra + 32 * src_w;
        uint64_t a[kSuper], b[kSuper];
#pragma unroll
        for (int k = 0; k < kSuper; ++k) {
            a[k] = k < nk ? ra[k] : 0;
            b[k] = k < nk ? rb[k] : 0;
        }
#pragma unroll
        for (int k = 0; k < kSuper; ++k) {
            if (k >= nk) break;
            uint64_t out_a = from_res ? to_interchange(a[k]) : a[k];
            uint64_t out_b = from_res ? to_interchange(b[k]) : b[k];
            transpose64_lanes(out_a, out_b);   // now output rows 64 tj + lane and 64 tj + 32 + lane
            sm[k][lane][w] = to_res ? to_resident(out_a) : out_a;
            sm[k][lane + 32][w] = to_res ? to_resident(out_b) : out_b;
        }
    }
    __syncthreads();
    const int64_t dst_w = nti;
    for (int idx = threadIdx.x; idx < kSuper * 64 * kSuper; idx += blockDim.x) {
        const int ww = idx % kSuper, r = (idx / kSuper) % 64, k = idx / (64 * kSuper);
        if (ww < nw && k < nk) dst[(64 * (kSuper * sj + k) + r) * dst_w + kSuper * si + ww] = sm[k][r][ww];
    }
}

// Transposed orientation, super-tile per block: the board (R rows, W words)
// to its stored transpose (to_res), or back.
__global__ void orient_super_kernel(const uint64_t *__restrict__ src, uint64_t *__restrict__ dst, int64_t R,
                                    int64_t W, bool to_res) {
    const int64_t src_rows = to_res ? R : 64 * W, src_w = to_res ? W : R / 64;
    const int64_t nsj = (src_w + kSuper - 1) / kSuper;
    transpose_super(src, src_rows, src_w, dst, blockIdx.x / nsj, blockIdx.x % nsj, !to_res, to_res);
}

// R x W interchange words <-> resident storage in the same orientation
// (transposed boards go through orient_super_kernel).
// last_bits (1..63): the last word of every row holds that many columns and
// its other bits are cleared on the way (0: whole words).
__global__ void orient_kernel(const uint64_t *__restrict__ src, uint64_t *__restrict__ dst, int64_t R, int64_t W,
                              bool to_res, int last_bits) {
    const int64_t n = R * W;
    const uint64_t keep = last_bits ? (1ull << last_bits) - 1 : ~0ull;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t w = src[i];
        const bool last = i % W == W - 1;
        if (to_res) {
            if (last) w &= keep;
            dst[i] = to_resident(w);
        } else {
            w = to_interchange(w);
            dst[i] = last ? (w & keep) : w;
        }
    }
}

// Rows of C cells -> rows of ceil(C / 64) words (interchange layout, padding
// zero); flags cell values other than 0 / 1.  One thread per word.
__global__ void pack_rows_kernel(const uint8_t *__restrict__ cells, uint64_t *__restrict__ words, int64_t R,
                                 int64_t C, int32_t *bad) {
    const int64_t W = (C + 63) / 64, n = R * W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / W, k = i - r * W;
        const uint8_t *p = cells + r * C + 64 * k;
        const int m = (int)min((int64_t)64, C - 64 * k);
        uint64_t w = 0;
        bool high = false;
        for (int j = 0; j < m; ++j) {
            const uint8_t v = p[j];
            high |= v > 1;
            w |= (uint64_t)(v & 1) << j;
        }
        if (high) atomicExch(bad, 1);
        words[i] = w;
    }
}

__global__ void unpack_rows_kernel(const uint64_t *__restrict__ words, uint8_t *__restrict__ cells, int64_t R,
                                   int64_t C) {
    const int64_t n = R * C, W = (C + 63) / 64;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / C, c = i - r * C;
        cells[i] = (uint8_t)((words[r * W + (c >> 6)] >> (c & 63)) & 1u);
    }
}

// --- many boards <-> one contiguous staging buffer ----------------------------
// The copy grid holds copy_blocks(d[i]) consecutive blocks per board;
// block_board maps a block to its board.  A block copies its share of the
// board's words, or one super-tile when the board is stored transposed.
__global__ void scatter_boards_kernel(const CopyDesc *__restrict__ d, const int32_t *__restrict__ block_board,
                                      const uint64_t *__restrict__ staging) {
    const CopyDesc c = d[block_board[blockIdx.x]];
    const int64_t lb = blockIdx.x - c.block0;
    if (!c.transposed) {
        const int64_t end = min(c.nwords, (lb + 1) * kCopyWordsPerBlock);
        const uint64_t keep = c.last_bits ? (1ull << c.last_bits) - 1 : ~0ull;
        for (int64_t i = lb * kCopyWordsPerBlock + threadIdx.x; i < end; i += blockDim.x) {
            uint64_t w = staging[c.offset + i];
            if (i % c.words == c.words - 1) w &= keep;
            c.buf[0][i] = to_resident(w);
        }
    } else {
        // super-tile lb of the board (rows x words interchange) -> its stored transpose
        const int64_t nsj = (c.words + kSuper - 1) / kSuper;
        transpose_super(staging + c.offset, c.rows, c.words, c.buf[0], lb / nsj, lb % nsj, false, true);
    }
    if (lb == 0 && threadIdx.x == 0) *c.cur = 0;
}

__global__ void gather_boards_kernel(const CopyDesc *__restrict__ d, const int32_t *__restrict__ block_board,
                                     uint64_t *__restrict__ staging) {
    const CopyDesc c = d[block_board[blockIdx.x]];
    const int64_t lb = blockIdx.x - c.block0;
    const uint64_t *board = c.buf[*c.cur & 1];
    if (!c.transposed) {
        const int64_t end = min(c.nwords, (lb + 1) * kCopyWordsPerBlock);
        for (int64_t i = lb * kCopyWordsPerBlock + threadIdx.x; i < end; i += blockDim.x)
            staging[c.offset + i] = to_interchange(board[i]);
    } else {
        // super-tile lb of the stored transpose (64 words x rows / 64) -> interchange rows
        const int64_t rb = c.rows / 64, nsj = (rb + kSuper - 1) / kSuper;
        transpose_super(board, 64 * c.words, rb, staging + c.offset, lb / nsj, lb % nsj, true, false);
    }
}

// --- integer-pipe probe -------------------------------------------------------
// Eight independent chains; per iteration and chain five LOP3 and one funnel
// shift, the 20:4 LOP3:SHF ratio of one generation of a word.
constexpr int kProbeChains = 8;
constexpr int kProbeOpsPerChain = 6;

__global__ void int_probe_kernel(unsigned *sink, int iters) {
    uint32_t x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = threadIdx.x * 0x9E3779B9u + c * 0x85EBCA6Bu + blockIdx.x;
    uint32_t y = threadIdx.x ^ 0x5bd1e995u, z = blockIdx.x ^ 0x27d4eb2fu;
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) {
            uint32_t v = x[c];
            v = lop3<0x96>(v, y, z);
            v = lop3<0xE8>(v, z, y);
            v = lop3<0x14>(v, y, z);
            v = __funnelshift_l(v, y, 1 + (c & 3));
            v = lop3<0x82>(v, z, y);
            v = lop3<0xCA>(v, y, z);
            x[c] = v;
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) acc ^= x[c];
    if (acc == 0x12345678u) sink[blockIdx.x] = acc;   // keeps the chains live
}

std::atomic<uint64_t> g_launch_count{0};
thread_local bool t_capturing = false;

}  // namespace

void count_launches(int n) {
    if (!t_capturing) g_launch_count.fetch_add((uint64_t)n, std::memory_order_relaxed);
}
void set_capturing(bool on) { t_capturing = on; }
uint64_t launches_so_far() { return g_launch_count.load(std::memory_order_relaxed); }

cudaError_t launch_sched_init(const PersistArgs &a, int nboards, cudaStream_t s) {
    const int64_t n = max(max((int64_t)a.nunits, (int64_t)a.total_tasks), (int64_t)max(nboards, 32));
    sched_init_kernel<<<grid_for(n, kBlock, 4096), kBlock, 0, s>>>(a, nboards);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_byte_step(const uint8_t *in, uint8_t *out, int64_t R, int64_t C, int torus,
                             cudaStream_t s) {
    byte_step_kernel<<<grid_for(R * C), kBlock, 0, s>>>(in, out, R, C, torus);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pack(const uint8_t *cells, uint64_t *words, int64_t R, int64_t W, int32_t *bad,
                        cudaStream_t s) {
    pack_kernel<<<grid_for(R * W), kBlock, 0, s>>>(cells, words, R * W, bad);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_check_bytes(const uint8_t *cells, int64_t n, int32_t *bad, cudaStream_t s) {
    check_bytes_kernel<<<grid_for(n), kBlock, 0, s>>>(cells, n, bad);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const uint64_t *words, uint8_t *cells, int64_t R, int64_t W, cudaStream_t s) {
    unpack_kernel<<<grid_for(R * W), kBlock, 0, s>>>(words, cells, R * W);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_region_packed(const uint64_t *words, int64_t R, int64_t C, int64_t r0, int64_t c0,
                                 int64_t nr, int64_t nc, uint8_t *out, bool transposed, cudaStream_t s) {
    region_packed_kernel<<<grid_for(nr * nc), kBlock, 0, s>>>(words, R, C, r0, c0, nr, nc, out, transposed);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pack_transposed(const uint8_t *cells, int64_t R, int64_t C, uint64_t *store, int32_t *bad,
                                   cudaStream_t s) {
    if (R * C > 0) pack_transposed_kernel<<<grid_for((R / 64) * C), kBlock, 0, s>>>(cells, R, C, store, bad);
    if (R * C > 0) count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_unpack_transposed(const uint64_t *store, int64_t R, int64_t C, uint8_t *cells, cudaStream_t s) {
    if (R * C > 0) unpack_transposed_kernel<<<grid_for((R / 64) * C), kBlock, 0, s>>>(store, R, C, cells);
    if (R * C > 0) count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pack_rows(const uint8_t *cells, uint64_t *words, int64_t R, int64_t C, int32_t *bad,
                             cudaStream_t s) {
    const int64_t n = R * ((C + 63) / 64);
    if (n > 0) pack_rows_kernel<<<grid_for(n), kBlock, 0, s>>>(cells, words, R, C, bad);
    if (n > 0) count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_unpack_rows(const uint64_t *words, uint8_t *cells, int64_t R, int64_t C, cudaStream_t s) {
    if (R * C > 0) unpack_rows_kernel<<<grid_for(R * C), kBlock, 0, s>>>(words, cells, R, C);
    if (R * C > 0) count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_orient(const uint64_t *src, uint64_t *dst, int64_t R, int64_t W, bool transposed, bool to_res,
                          cudaStream_t s, int last_bits) {
    if (R * W == 0) return cudaSuccess;
    if (transposed) {
        const int64_t nsuper = ((R / 64 + kSuper - 1) / kSuper) * ((W + kSuper - 1) / kSuper);
        orient_super_kernel<<<(unsigned)nsuper, kBlock, 0, s>>>(src, dst, R, W, to_res);
        count_launches(1);
    } else {
        orient_kernel<<<grid_for(R * W, kBlock, 1 << 16), kBlock, 0, s>>>(src, dst, R, W, to_res, last_bits);
        count_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t launch_region_bytes(const uint8_t *cells, int64_t R, int64_t C, int64_t r0, int64_t c0,
                                int64_t nr, int64_t nc, uint8_t *out, cudaStream_t s) {
    region_bytes_kernel<<<grid_for(nr * nc), kBlock, 0, s>>>(cells, R, C, r0, c0, nr, nc, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_popcount_packed(const uint64_t *words, int64_t n, unsigned long long *out,
                                   cudaStream_t s) {
    popcount_kernel<uint64_t><<<grid_for(n, kBlock, 8192), kBlock, 0, s>>>(words, n, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_popcount_bytes(const uint8_t *cells, int64_t n, unsigned long long *out,
                                  cudaStream_t s) {
    popcount_kernel<uint8_t><<<grid_for(n, kBlock, 8192), kBlock, 0, s>>>(cells, n, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_convert(const uint64_t *src, uint64_t *dst, int64_t n, bool to_res, cudaStream_t s) {
    if (n > 0) convert_kernel<<<grid_for(n, kBlock, 1 << 16), kBlock, 0, s>>>(src, dst, n, to_res);
    if (n > 0) count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_scatter_boards(const CopyDesc *d, const int32_t *block_board, int64_t blocks, const uint64_t *staging,
                                  cudaStream_t s) {
    if (blocks > 0) scatter_boards_kernel<<<(unsigned)blocks, kBlock, 0, s>>>(d, block_board, staging);
    if (blocks > 0) count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gather_boards(const CopyDesc *d, const int32_t *block_board, int64_t blocks, uint64_t *staging,
                                 cudaStream_t s) {
    if (blocks > 0) gather_boards_kernel<<<(unsigned)blocks, kBlock, 0, s>>>(d, block_board, staging);
    if (blocks > 0) count_launches(1);
    return cudaGetLastError();
}

int byte_cluster_size(int64_t R, int64_t C) {
    if (R < 1 || C < 1 || R > (1 << 20) || C > (1 << 20)) return 0;
    const int64_t W = (C + 63) / 64;
    for (int n = 1; n <= kByteClusterMax && n <= R; n *= 2) {
        const int64_t hmax = (R + n - 1) / n;
        if (2 * hmax * W * 8 <= kByteClusterBytes) return n;
    }
    return 0;
}

// Cluster size used for a board: `want` when it is a power of two <= 8 that
// fits (forced), else the smallest power of two that fits and leaves each CTA
// at most kByteWordsPerCta words (more CTAs share the generation's work).
int byte_cluster_choice(int64_t R, int64_t C, int want) {
    const int nmin = byte_cluster_size(R, C);
    if (nmin == 0) return 0;
    const int64_t W = (C + 63) / 64;
    if (want > 1) {
        if ((want & (want - 1)) || want > kByteClusterMax || want > R || want < nmin) return nmin;
        return want;
    }
    int n = nmin;
    while (n < kByteClusterMax && 2 * n <= R && ((R + n - 1) / n) * W > kByteWordsPerCta) n *= 2;
    return n;
}

cudaError_t launch_byte_cluster(const uint8_t *in, uint8_t *out, int64_t R, int64_t C, int torus, int G, int want,
                                cudaStream_t s) {
    const int n = byte_cluster_choice(R, C, want);
    if (n == 0 || G < 1) return cudaErrorInvalidValue;
    const int64_t hmax = (R + n - 1) / n, W = (C + 63) / 64;
    const size_t smem = (size_t)(2 * hmax * W * 8);
    // one thread per word of a strip, in whole warps, 64 .. 1024
    const unsigned threads = (unsigned)std::min<int64_t>(1024, std::max<int64_t>(64, (hmax * W + 31) / 32 * 32));
    if (n == 1) {
        cudaError_t e = cudaFuncSetAttribute(byte_resident_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        byte_resident_kernel<false><<<1, threads, smem, s>>>(in, out, (int)R, (int)C, torus, G);
        count_launches(1);
        return cudaGetLastError();
    }
    cudaError_t e = cudaFuncSetAttribute(byte_resident_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)n, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)n;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, byte_resident_kernel<true>, in, out, (int)R, (int)C, torus, G);
    if (e == cudaSuccess) count_launches(1);
    return e;
}

cudaError_t launch_int_probe(unsigned *sink, int iters, int grid, int block, cudaStream_t s) {
    int_probe_kernel<<<grid, block, 0, s>>>(sink, iters);
    count_launches(1);
    return cudaGetLastError();
}

int int_probe_ops_per_iter() { return kProbeChains * kProbeOpsPerChain; }

}  // namespace gol
