// Packed Game of Life step: a register wavefront over bit-sliced words,
// run by a persistent dataflow scheduler.
//
// Arithmetic (Section 1 of the paper).  A lane holds one 64-cell word of a
// row in the resident layout (low half = even columns, high half = odd
// columns, see gol_internal.h).  For an input row it forms the row's
// horizontal three-cell sum per column as two bit planes:
//     Wv = the west neighbour of every column, Ev = the east neighbour; for
//          the even half they are the odd half shifted by one (carry bit from
//          the west word, fetched from the neighbouring lane) and the odd half
//          itself, for the odd half the even half itself and the even half
//          shifted by one (carry from the east word)
//     s0 = Wv ^ x ^ Ev,  s1 = majority(Wv, x, Ev)          (s = s0 + 2 s1)
// The nine-cell sum of a cell is S = s(row above) + s(row) + s(row below),
// which includes the cell itself, so with n = S - alive the four
// transitions reduce to  next = (S == 3) | (alive & (S == 4)).  That
// predicate is evaluated bit-sliced with eight 3-input LOP3 operations per
// 32-bit half (rule32).  One generation of a word costs 2 funnel shifts +
// 20 LOP3 = 22 integer operations and 2 warp shuffles.
//
// Temporal blocking.  A warp streams the rows of its unit top to bottom
// through K pipeline stages held in registers; stage g turns generation g
// rows into generation g+1 rows, keeping a three-row window (two row sums
// and one alive word).  A unit with H output rows per segment reads
// H + 2K input rows of the previous buffer (a K-row halo above and below,
// taken modulo R on the torus) and writes H rows of generation kk <= K.
// Stages g >= kk pass rows through unchanged, so one kernel serves passes
// of any length up to K.  Horizontally the validity of a tiled warp shrinks
// by one cell per generation from each side, so one halo word per side is
// exact for K <= 64.
//
// Scheduling.  A unit's pass p reads pass p-1 output of every unit whose
// output its halo touches (its neighbours) and overwrites the buffer those
// units read during pass p-1; it may start once all of them have completed
// pass p-1.  After a pass a warp counts down the join counter of u and of
// each neighbour (complete_pass): the finisher that empties a counter claims
// that unit and either runs it next in the same warp or queues it.  Queued
// passes wait in two rings, critical (much of the unit's chain still ahead)
// and the rest; warps take slots by atomicAdd tickets only and serve the
// critical ring first (take_work).  Every wait is bounded: a waiter gives up
// after `timeout_ns` without any task completing, records GOL_ETIMEOUT and
// returns.
#pragma once

#include <type_traits>

#include "gol_internal.h"

// 1: the guarded prologue iterations of a pass are unrolled completely.
#ifndef GOL_UNROLL_PROLOGUE
#define GOL_UNROLL_PROLOGUE 1
#endif

namespace gol {

template <unsigned LUT>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
    return d;
}

// LUT constants: f(0xF0, 0xCC, 0xAA) for operands (a, b, c).
constexpr unsigned kXor3 = 0x96;   // a ^ b ^ c
constexpr unsigned kMaj3 = 0xE8;   // majority(a, b, c)

// Next state of 32 cells from the row-sum planes of the rows above (t),
// at (m) and below (b) and the alive bits a of the middle row.
//   t0+m0+b0 = u0 + 2 u1,  t1+m1+b1 = p + 2 q  =>  S = u0 + 2 (u1 + p) + 4 q
//   S == 3      <=> u0 & (p ^ u1) & ~q
//   S == 4      <=> ~u0 & ~(p ^ u1) & (p ^ q)
__device__ __forceinline__ uint32_t rule32(uint32_t t0, uint32_t t1, uint32_t m0, uint32_t m1,
                                           uint32_t b0, uint32_t b1, uint32_t a) {
    const uint32_t u0 = lop3<kXor3>(t0, m0, b0);
    const uint32_t u1 = lop3<kMaj3>(t0, m0, b0);
    const uint32_t p = lop3<kXor3>(t1, m1, b1);
    const uint32_t q = lop3<kMaj3>(t1, m1, b1);
    const uint32_t x3 = lop3<0x14>(p, u1, q);   // (p ^ u1) & ~q
    const uint32_t y1 = lop3<0x82>(p, u1, a);   // ~(p ^ u1) & a
    const uint32_t y4 = lop3<0x60>(y1, p, q);   // y1 & (p ^ q)
    return lop3<0xCA>(u0, x3, y4);              // u0 ? x3 : y4
}

// ---------------------------------------------------------------------------
// memory-model helpers (PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ld_acquire(const int32_t *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int32_t *p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint2 ld_cg_u64(const uint64_t *p) {
    uint2 v;
    asm volatile("ld.global.cg.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ void st_u64(uint64_t *p, uint32_t lo, uint32_t hi) {
    asm volatile("st.global.v2.u32 [%0], {%1, %2};" ::"l"(p), "r"(lo), "r"(hi) : "memory");
}

// ---------------------------------------------------------------------------
// One pass of one unit by one warp.
// ---------------------------------------------------------------------------
// Variant of run_unit_pass whose three-row window shifts by register moves
// (iteration loop unrolled twice); fewer registers, more issue slots.
template <int K, bool TORUS, bool PARTIAL>
__device__ __forceinline__ void run_unit_pass_moves(const UnitRun &ud,
                                              const uint64_t *__restrict__ src,
                                              uint64_t *__restrict__ dst, int kk) {
    constexpr unsigned kFull = 0xffffffffu;
    constexpr int PF = 2;                          // rows prefetched ahead (2K is a multiple)
    constexpr int NPRO = 2 * K;                    // prologue iterations
    const int lane = threadIdx.x & 31;
    const int R = ud.R, W = ud.W;

    // ---- lane geometry -------------------------------------------------
    int seg = 0, word = 0, west_src = lane, east_src = lane;
    bool loads = false, stores = false;
    uint32_t west_mask = ~0u, east_mask = ~0u, lane_mask = ~0u;
    if ((ud.mode & 0xff) == kUnitFull) {
        seg = lane / W;
        word = lane - seg * W;
        if (seg < ud.S) {
            loads = stores = true;
            const int base = lane - word;
            west_src = base + (word == 0 ? W - 1 : word - 1);
            east_src = base + (word == W - 1 ? 0 : word + 1);
            if (!TORUS) {
                if (word == 0) west_mask = 0;
                if (word == W - 1) east_mask = 0;
            }
        } else {
            seg = 0;
            word = 0;
        }
    } else {
        int w = ud.w0 - 1 + lane;
        loads = lane < ud.U + 2;
        stores = lane >= 1 && lane <= ud.U;
        if (TORUS) {
            w = w < 0 ? w + W : (w >= W ? w - W : w);
        } else if (w < 0 || w >= W) {
            lane_mask = 0;
            loads = false;
            w = 0;
        }
        word = loads ? w : 0;
        west_src = lane == 0 ? 0 : lane - 1;
        east_src = lane == 31 ? 31 : lane + 1;
    }
    const int a = ud.r0 + seg * ud.H;                       // first output row of the segment
    const int seg_end = min(a + ud.H, ud.r_end);            // one past its last output row
    const int nmain = ud.H;                                 // main-loop iterations

    // ---- input row stream: row (a - K + j) of src ---------------------
    int lrow = a - K;                                       // row of the next load (unwrapped)
    int lwrap = lrow;                                       // wrapped row
    if (TORUS) {
        lwrap %= R;
        if (lwrap < 0) lwrap += R;
    }
    const uint64_t *colp = src + word;
    auto load_next = [&](uint32_t &lo, uint32_t &hi) {
        lo = hi = 0;
        if (TORUS) {
            if (loads) {
                const uint2 v = ld_cg_u64(colp + (size_t)lwrap * W);
                lo = v.x;
                hi = v.y;
            }
            if (++lwrap == R) lwrap = 0;
        } else {
            if (loads && lrow >= 0 && lrow < R) {
                const uint2 v = ld_cg_u64(colp + (size_t)lrow * W);
                lo = v.x;
                hi = v.y;
            }
        }
        ++lrow;
    };

    // ---- pipeline registers ----------------------------------------------
    uint32_t p0l[K], p0h[K], p1l[K], p1h[K];   // row sum two rows back
    uint32_t c0l[K], c0h[K], c1l[K], c1h[K];   // row sum one row back
    uint32_t cal[K], cah[K];                   // alive word one row back
#pragma unroll
    for (int g = 0; g < K; ++g) {
        p0l[g] = p0h[g] = p1l[g] = p1h[g] = 0;
        c0l[g] = c0h[g] = c1l[g] = c1h[g] = 0;
        cal[g] = cah[g] = 0;
    }
    uint32_t fl[PF], fh[PF];
#pragma unroll
    for (int u = 0; u < PF; ++u) load_next(fl[u], fh[u]);

    // One iteration: the gen-0 row (a - K + j) enters stage 0; returns the
    // generation-kk row (a + j - 2K) leaving the last stage.  In the
    // prologue (GUARD) stage g only runs once its window holds valid rows.
    auto iterate = [&](uint32_t xl, uint32_t xh, int j, auto guard_tag) {
        constexpr bool GUARD = decltype(guard_tag)::value;
        const int jr = a - K + j;
#pragma unroll
        for (int g = 0; g < K; ++g) {
            if (GUARD && j < 2 * g) break;                  // input of stage g not produced yet
            const uint32_t wh = __shfl_sync(kFull, xh, west_src) & west_mask;
            const uint32_t el = __shfl_sync(kFull, xl, east_src) & east_mask;
            // even columns (low half): west = odd column to the left = the
            // high half shifted up by one, its bit 0 from the west word;
            // east = the odd column to the right = the high half as is.
            // odd columns (high half): west = the low half as is; east = the
            // low half shifted down by one, its bit 31 from the east word.
            const uint32_t Wl = __funnelshift_l(wh, xh, 1);
            const uint32_t Eh = __funnelshift_r(xl, el, 1);
            const uint32_t n0l = lop3<kXor3>(Wl, xl, xh), n0h = lop3<kXor3>(xl, xh, Eh);
            const uint32_t n1l = lop3<kMaj3>(Wl, xl, xh), n1h = lop3<kMaj3>(xl, xh, Eh);
            uint32_t ol = 0, oh = 0;
            if (!GUARD || j >= 2 * g + 2) {
                ol = rule32(p0l[g], p1l[g], c0l[g], c1l[g], n0l, n1l, cal[g]);
                oh = rule32(p0h[g], p1h[g], c0h[g], c1h[g], n0h, n1h, cah[g]);
                if (PARTIAL && g >= kk) {                   // pass shorter than K: identity stage
                    ol = cal[g];
                    oh = cah[g];
                }
                if (!TORUS) {
                    const bool inside = (unsigned)(jr - g - 1) < (unsigned)R;
                    ol = inside ? (ol & lane_mask) : 0u;
                    oh = inside ? (oh & lane_mask) : 0u;
                }
            }
            p0l[g] = c0l[g];
            p0h[g] = c0h[g];
            p1l[g] = c1l[g];
            p1h[g] = c1h[g];
            c0l[g] = n0l;
            c0h[g] = n0h;
            c1l[g] = n1l;
            c1h[g] = n1h;
            cal[g] = xl;
            cah[g] = xh;
            xl = ol;
            xh = oh;
        }
        return make_uint2(xl, xh);
    };

#pragma unroll 1
    for (int j0 = 0; j0 < NPRO; j0 += PF) {
#pragma unroll
        for (int u = 0; u < PF; ++u) {
            const uint32_t xl = fl[u], xh = fh[u];
            load_next(fl[u], fh[u]);
            iterate(xl, xh, j0 + u, std::true_type{});
        }
    }
    int orow = a;                                           // row of the next output
    uint64_t *outp = dst + word;
#pragma unroll 1
    for (int j0 = 0; j0 < nmain; j0 += PF) {
#pragma unroll
        for (int u = 0; u < PF; ++u) {
            const uint32_t xl = fl[u], xh = fh[u];
            load_next(fl[u], fh[u]);
            const uint2 o = iterate(xl, xh, NPRO + j0 + u, std::false_type{});
            if (stores && orow < seg_end) st_u64(outp + (size_t)orow * W, o.x, o.y);
            ++orow;
        }
    }
}


// Variant whose window slots rotate by renaming (loop unrolled three times).
//
// MASKED: a board whose width C is not a multiple of 64, stored with
// ceil(C / 64) words per row, the last word holding C' = C mod 64 columns
// (ud.mode >> 8) and zero padding above them.  In every stage the lane that
// holds the last word (a) writes column 0's state (the east word's bit 0,
// zero on a bounded board) into the first padding column, which is then the
// east neighbour of column C - 1, and (b) sends word 0's lane a value whose
// bit 31 is column C - 1, its west neighbour across the wrap.  No real cell
// has any other padding cell as a neighbour, so the padding needs no other
// care inside a pass; stored rows have their padding cleared.
template <int K, bool TORUS, bool PARTIAL, bool MASKED = false>
__device__ __forceinline__ void run_unit_pass(const UnitRun &ud,
                                              const uint64_t *__restrict__ src,
                                              uint64_t *__restrict__ dst, int kk) {
    constexpr unsigned kFull = 0xffffffffu;
    constexpr int NPRO = 2 * K;                    // iterations before the first output row
    constexpr int NPRO3 = (NPRO + 2) / 3 * 3;      // guarded iterations (multiple of 3)
    const int lane = threadIdx.x & 31;
    const int R = ud.R, W = ud.W;

    // ---- lane geometry -------------------------------------------------
    int seg = 0, word = 0, west_src = lane, east_src = lane;
    bool loads = false, stores = false;
    uint32_t west_mask = ~0u, east_mask = ~0u, lane_mask = ~0u;
    if ((ud.mode & 0xff) == kUnitFull) {
        seg = lane / W;
        word = lane - seg * W;
        if (seg < ud.S) {
            loads = stores = true;
            const int base = lane - word;
            west_src = base + (word == 0 ? W - 1 : word - 1);
            east_src = base + (word == W - 1 ? 0 : word + 1);
            if (!TORUS) {
                if (word == 0) west_mask = 0;
                if (word == W - 1) east_mask = 0;
            }
        } else {
            seg = 0;
            word = 0;
        }
    } else {
        int w = ud.w0 - 1 + lane;
        loads = lane < ud.U + 2;
        stores = lane >= 1 && lane <= ud.U;
        if (TORUS) {
            w = w < 0 ? w + W : (w >= W ? w - W : w);
        } else if (w < 0 || w >= W) {
            lane_mask = 0;
            loads = false;
            w = 0;
        }
        word = loads ? w : 0;
        west_src = lane == 0 ? 0 : lane - 1;
        east_src = lane == 31 ? 31 : lane + 1;
    }
    const int a = ud.r0 + seg * ud.H;                       // first output row of the segment
    const int seg_end = min(a + ud.H, ud.r_end);            // one past its last output row
    const int nmain = ud.H;                                 // main-loop iterations

    // ---- masked last word (see above) --------------------------------
    // last lane: pad_shift / pad_l / pad_h place column 0's bit at the first
    // padding column (even C': low half bit C'/2, odd C': high half bit
    // (C'-1)/2); west_n / west_pick make bit 31 of the value sent west
    // column C - 1 (even C': high half bit C'/2 - 1, odd C': low half bit
    // (C'-1)/2); keep_l / keep_h clear the padding of stored words.  Other
    // lanes: all masks zero, west_n = 0 (they send their high half).
    uint32_t pad_shift = 0, pad_l = 0, pad_h = 0, west_n = 0, west_pick = 0, keep_l = ~0u, keep_h = ~0u;
    bool warp_last = false;                                 // some lane of this warp holds word W - 1
    if (MASKED) {
        const int cl = (ud.mode >> 8) & 0xff;               // valid columns of the last word, 1 .. 63
        warp_last = __ballot_sync(kFull, loads && word == W - 1) != 0;
        if (loads && word == W - 1) {
            pad_shift = (uint32_t)(cl >> 1);
            if (cl & 1)
                pad_h = 1u << pad_shift;
            else
                pad_l = 1u << pad_shift;
            west_n = (uint32_t)((cl + 1) >> 1);
            west_pick = (cl & 1) ? ~0u : 0u;
            keep_l = ((cl + 1) >> 1) >= 32 ? ~0u : (1u << ((cl + 1) >> 1)) - 1u;
            keep_h = (1u << (cl >> 1)) - 1u;
        }
    }

    // ---- input row stream: row (a - K + j) of src ---------------------
    int lrow = a - K;                                       // row of the next load (unwrapped)
    int lwrap = lrow;                                       // wrapped row
    if (TORUS) {
        lwrap %= R;
        if (lwrap < 0) lwrap += R;
    }
    const uint64_t *colp = src + word;
    auto load_next = [&](uint32_t &lo, uint32_t &hi) {
        lo = hi = 0;
        if (TORUS) {
            if (loads) {
                const uint2 v = ld_cg_u64(colp + (size_t)lwrap * W);
                lo = v.x;
                hi = v.y;
            }
            if (++lwrap == R) lwrap = 0;
        } else {
            if (loads && lrow >= 0 && lrow < R) {
                const uint2 v = ld_cg_u64(colp + (size_t)lrow * W);
                lo = v.x;
                hi = v.y;
            }
        }
        ++lrow;
    };

    // ---- pipeline registers ----------------------------------------------
    // Each stage keeps three row slots (row-sum planes and alive word) that
    // take the roles (two rows back, one row back, current row) in turn: the
    // iteration loop is unrolled three times so that the roles rotate by
    // renaming instead of register moves.
    uint32_t s0l[3][K], s0h[3][K], s1l[3][K], s1h[3][K], sal[3][K], sah[3][K];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int g = 0; g < K; ++g) s0l[r][g] = s0h[r][g] = s1l[r][g] = s1h[r][g] = sal[r][g] = sah[r][g] = 0;
    uint32_t fl[3], fh[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) load_next(fl[u], fh[u]);

    // One iteration: the gen-0 row (a - K + j) enters stage 0; returns the
    // generation-kk row (a + j - 2K) leaving the last stage.  PH = j mod 3
    // names the slot of the oldest row.  In the prologue (GUARD) stage g only
    // runs once its window holds valid rows.
    auto iterate = [&](uint32_t xl, uint32_t xh, int j, auto guard_tag, auto phase_tag) {
        constexpr bool GUARD = decltype(guard_tag)::value;
        constexpr int O = decltype(phase_tag)::value, M = (O + 1) % 3, N = (O + 2) % 3;
        const int jr = a - K + j;
#pragma unroll
        for (int g = 0; g < K; ++g) {
            if (GUARD && j < 2 * g) break;                  // input of stage g not produced yet
            // (warp_last is uniform over the warp: warps without the partial
            // word, all tiles but one of a wide board, skip the masked steps)
            uint32_t wsend = xh;
            if (MASKED && warp_last)
                wsend = __funnelshift_rc(xh, lop3<0xD8>(xh, xl, west_pick), west_n);   // shift 32: the high word
            const uint32_t wh = __shfl_sync(kFull, wsend, west_src) & west_mask;
            const uint32_t el = __shfl_sync(kFull, xl, east_src) & east_mask;
            if (MASKED && warp_last) {
                const uint32_t t = el << pad_shift;
                xl = lop3<0xD8>(xl, t, pad_l);              // pad_l ? t : xl, bit by bit
                xh = lop3<0xD8>(xh, t, pad_h);
            }
            // even columns (low half): west = odd column to the left = the
            // high half shifted up by one, its bit 0 from the west word;
            // east = the odd column to the right = the high half as is.
            // odd columns (high half): west = the low half as is; east = the
            // low half shifted down by one, its bit 31 from the east word.
            const uint32_t Wl = __funnelshift_l(wh, xh, 1);
            const uint32_t Eh = __funnelshift_r(xl, el, 1);
            s0l[N][g] = lop3<kXor3>(Wl, xl, xh);
            s0h[N][g] = lop3<kXor3>(xl, xh, Eh);
            s1l[N][g] = lop3<kMaj3>(Wl, xl, xh);
            s1h[N][g] = lop3<kMaj3>(xl, xh, Eh);
            sal[N][g] = xl;
            sah[N][g] = xh;
            uint32_t ol = 0, oh = 0;
            if (!GUARD || j >= 2 * g + 2) {
                ol = rule32(s0l[O][g], s1l[O][g], s0l[M][g], s1l[M][g], s0l[N][g], s1l[N][g], sal[M][g]);
                oh = rule32(s0h[O][g], s1h[O][g], s0h[M][g], s1h[M][g], s0h[N][g], s1h[N][g], sah[M][g]);
                if (PARTIAL && g >= kk) {                   // pass shorter than K: identity stage
                    ol = sal[M][g];
                    oh = sah[M][g];
                }
                if (!TORUS) {
                    const bool inside = (unsigned)(jr - g - 1) < (unsigned)R;
                    ol = inside ? (ol & lane_mask) : 0u;
                    oh = inside ? (oh & lane_mask) : 0u;
                }
            }
            xl = ol;
            xh = oh;
        }
        return make_uint2(xl, xh);
    };

    using P0 = std::integral_constant<int, 0>;
    using P1 = std::integral_constant<int, 1>;
    using P2 = std::integral_constant<int, 2>;
    int orow = a;                                           // row of the next output
    uint64_t *outp = dst + word;
    auto emit = [&](uint2 o) {
        if (MASKED) {
            o.x &= keep_l;
            o.y &= keep_h;
        }
        if (stores && orow < seg_end) st_u64(outp + (size_t)orow * W, o.x, o.y);
        ++orow;
    };
    // prologue: the first 2K iterations (rounded up to a multiple of 3) with
    // guards; iterations from 2K on already produce output rows.  Unrolled
    // completely, the guards are known at compile time and the partial
    // stages of successive iterations overlap.
#if GOL_UNROLL_PROLOGUE
#pragma unroll
#else
#pragma unroll 1
#endif
    for (int j0 = 0; j0 < NPRO3; j0 += 3) {
        uint32_t xl = fl[0], xh = fh[0];
        load_next(fl[0], fh[0]);
        uint2 o = iterate(xl, xh, j0, std::true_type{}, P0{});
        if (j0 >= NPRO) emit(o);
        xl = fl[1], xh = fh[1];
        load_next(fl[1], fh[1]);
        o = iterate(xl, xh, j0 + 1, std::true_type{}, P1{});
        if (j0 + 1 >= NPRO) emit(o);
        xl = fl[2], xh = fh[2];
        load_next(fl[2], fh[2]);
        o = iterate(xl, xh, j0 + 2, std::true_type{}, P2{});
        if (j0 + 2 >= NPRO) emit(o);
    }
#pragma unroll 1
    for (int j0 = NPRO3; j0 < NPRO + nmain; j0 += 3) {
        uint32_t xl = fl[0], xh = fh[0];
        load_next(fl[0], fh[0]);
        emit(iterate(xl, xh, j0, std::false_type{}, P0{}));
        xl = fl[1], xh = fh[1];
        load_next(fl[1], fh[1]);
        emit(iterate(xl, xh, j0 + 1, std::false_type{}, P1{}));
        xl = fl[2], xh = fh[2];
        load_next(fl[2], fh[2]);
        emit(iterate(xl, xh, j0 + 2, std::false_type{}, P2{}));
    }
}

// Variant with skewed stages: stage g > 0 takes the row that stage g - 1
// produced in the previous iteration (one register pair per stage boundary),
// so the K stages of an iteration do not depend on one another and their
// shuffle / funnel-shift / LOP3 chains overlap.  Each stage then delays the
// stream by two rows instead of one: stage g's output in iteration j is the
// generation-(g+1) row a - K + j - (2g + 1), the first output row a leaves
// in iteration 3K - 1, and a pass runs H + 3K - 1 iterations.  Window slots
// rotate by renaming as in run_unit_pass.
template <int K, bool TORUS, bool PARTIAL>
__device__ __forceinline__ void run_unit_pass_skew(const UnitRun &ud,
                                                   const uint64_t *__restrict__ src,
                                                   uint64_t *__restrict__ dst, int kk) {
    constexpr unsigned kFull = 0xffffffffu;
    constexpr int NOUT = 3 * K - 1;                // first iteration with an output row
    constexpr int NPRO3 = (NOUT + 2) / 3 * 3;      // guarded iterations (multiple of 3)
    const int lane = threadIdx.x & 31;
    const int R = ud.R, W = ud.W;

    // ---- lane geometry -------------------------------------------------
    int seg = 0, word = 0, west_src = lane, east_src = lane;
    bool loads = false, stores = false;
    uint32_t west_mask = ~0u, east_mask = ~0u, lane_mask = ~0u;
    if ((ud.mode & 0xff) == kUnitFull) {
        seg = lane / W;
        word = lane - seg * W;
        if (seg < ud.S) {
            loads = stores = true;
            const int base = lane - word;
            west_src = base + (word == 0 ? W - 1 : word - 1);
            east_src = base + (word == W - 1 ? 0 : word + 1);
            if (!TORUS) {
                if (word == 0) west_mask = 0;
                if (word == W - 1) east_mask = 0;
            }
        } else {
            seg = 0;
            word = 0;
        }
    } else {
        int w = ud.w0 - 1 + lane;
        loads = lane < ud.U + 2;
        stores = lane >= 1 && lane <= ud.U;
        if (TORUS) {
            w = w < 0 ? w + W : (w >= W ? w - W : w);
        } else if (w < 0 || w >= W) {
            lane_mask = 0;
            loads = false;
            w = 0;
        }
        word = loads ? w : 0;
        west_src = lane == 0 ? 0 : lane - 1;
        east_src = lane == 31 ? 31 : lane + 1;
    }
    const int a = ud.r0 + seg * ud.H;                       // first output row of the segment
    const int seg_end = min(a + ud.H, ud.r_end);            // one past its last output row
    const int nmain = ud.H;                                 // output rows per segment

    // ---- input row stream: row (a - K + j) of src ---------------------
    // (the last K - 1 iterations load rows past the unit's input; on the
    // torus they wrap, otherwise rows outside the board read as zero)
    int lrow = a - K;                                       // row of the next load (unwrapped)
    int lwrap = lrow;                                       // wrapped row
    if (TORUS) {
        lwrap %= R;
        if (lwrap < 0) lwrap += R;
    }
    const uint64_t *colp = src + word;
    auto load_next = [&](uint32_t &lo, uint32_t &hi) {
        lo = hi = 0;
        if (TORUS) {
            if (loads) {
                const uint2 v = ld_cg_u64(colp + (size_t)lwrap * W);
                lo = v.x;
                hi = v.y;
            }
            if (++lwrap == R) lwrap = 0;
        } else {
            if (loads && lrow >= 0 && lrow < R) {
                const uint2 v = ld_cg_u64(colp + (size_t)lrow * W);
                lo = v.x;
                hi = v.y;
            }
        }
        ++lrow;
    };

    // ---- pipeline registers ----------------------------------------------
    uint32_t s0l[3][K], s0h[3][K], s1l[3][K], s1h[3][K], sal[3][K], sah[3][K];
    uint32_t inl[K], inh[K];                   // inl[g]: stage g - 1's output of the last iteration
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int g = 0; g < K; ++g) s0l[r][g] = s0h[r][g] = s1l[r][g] = s1h[r][g] = sal[r][g] = sah[r][g] = 0;
#pragma unroll
    for (int g = 0; g < K; ++g) inl[g] = inh[g] = 0;
    uint32_t fl[3], fh[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) load_next(fl[u], fh[u]);

    // One iteration j: the gen-0 row (a - K + j) enters stage 0, every stage
    // g > 0 takes inl/inh[g]; returns the last stage's output, the
    // generation-kk row a + j - NOUT.  In the prologue (GUARD) stage g only
    // runs from iteration 3g on, when its input is a row of the unit.
    auto iterate = [&](uint32_t x0l, uint32_t x0h, int j, auto guard_tag, auto phase_tag) {
        constexpr bool GUARD = decltype(guard_tag)::value;
        constexpr int O = decltype(phase_tag)::value, M = (O + 1) % 3, N = (O + 2) % 3;
        uint32_t outl[K], outh[K];
#pragma unroll
        for (int g = 0; g < K; ++g) {
            outl[g] = outh[g] = 0;
            if (GUARD && j < 3 * g) continue;               // input of stage g not produced yet
            const uint32_t xl = g == 0 ? x0l : inl[g], xh = g == 0 ? x0h : inh[g];
            const uint32_t wh = __shfl_sync(kFull, xh, west_src) & west_mask;
            const uint32_t el = __shfl_sync(kFull, xl, east_src) & east_mask;
            const uint32_t Wl = __funnelshift_l(wh, xh, 1);
            const uint32_t Eh = __funnelshift_r(xl, el, 1);
            s0l[N][g] = lop3<kXor3>(Wl, xl, xh);
            s0h[N][g] = lop3<kXor3>(xl, xh, Eh);
            s1l[N][g] = lop3<kMaj3>(Wl, xl, xh);
            s1h[N][g] = lop3<kMaj3>(xl, xh, Eh);
            sal[N][g] = xl;
            sah[N][g] = xh;
            uint32_t ol = rule32(s0l[O][g], s1l[O][g], s0l[M][g], s1l[M][g], s0l[N][g], s1l[N][g], sal[M][g]);
            uint32_t oh = rule32(s0h[O][g], s1h[O][g], s0h[M][g], s1h[M][g], s0h[N][g], s1h[N][g], sah[M][g]);
            if (PARTIAL && g >= kk) {                       // pass shorter than K: identity stage
                ol = sal[M][g];
                oh = sah[M][g];
            }
            if (!TORUS) {
                const bool inside = (unsigned)(a - K + j - 2 * g - 1) < (unsigned)R;
                ol = inside ? (ol & lane_mask) : 0u;
                oh = inside ? (oh & lane_mask) : 0u;
            }
            outl[g] = ol;
            outh[g] = oh;
        }
#pragma unroll
        for (int g = 1; g < K; ++g) {
            inl[g] = outl[g - 1];
            inh[g] = outh[g - 1];
        }
        return make_uint2(outl[K - 1], outh[K - 1]);
    };

    using P0 = std::integral_constant<int, 0>;
    using P1 = std::integral_constant<int, 1>;
    using P2 = std::integral_constant<int, 2>;
    int orow = a;                                           // row of the next output
    uint64_t *outp = dst + word;
    auto emit = [&](uint2 o) {
        if (stores && orow < seg_end) st_u64(outp + (size_t)orow * W, o.x, o.y);
        ++orow;
    };
#if GOL_UNROLL_PROLOGUE
#pragma unroll
#else
#pragma unroll 1
#endif
    for (int j0 = 0; j0 < NPRO3; j0 += 3) {
        uint32_t xl = fl[0], xh = fh[0];
        load_next(fl[0], fh[0]);
        uint2 o = iterate(xl, xh, j0, std::true_type{}, P0{});
        if (j0 >= NOUT) emit(o);
        xl = fl[1], xh = fh[1];
        load_next(fl[1], fh[1]);
        o = iterate(xl, xh, j0 + 1, std::true_type{}, P1{});
        if (j0 + 1 >= NOUT) emit(o);
        xl = fl[2], xh = fh[2];
        load_next(fl[2], fh[2]);
        o = iterate(xl, xh, j0 + 2, std::true_type{}, P2{});
        if (j0 + 2 >= NOUT) emit(o);
    }
#pragma unroll 1
    for (int j0 = NPRO3; j0 < NOUT + nmain; j0 += 3) {
        uint32_t xl = fl[0], xh = fh[0];
        load_next(fl[0], fh[0]);
        emit(iterate(xl, xh, j0, std::false_type{}, P0{}));
        xl = fl[1], xh = fh[1];
        load_next(fl[1], fh[1]);
        emit(iterate(xl, xh, j0 + 1, std::false_type{}, P1{}));
        xl = fl[2], xh = fh[2];
        load_next(fl[2], fh[2]);
        emit(iterate(xl, xh, j0 + 2, std::false_type{}, P2{}));
    }
}

// ---------------------------------------------------------------------------
// Scheduler
// ---------------------------------------------------------------------------
// Generations of pass `pass` (1-based) of a unit.  Without a population
// trace the board's generations are spread over its passes, the first
// ones one longer.  With a trace (ppp > 0) the launch is npass / ppp
// sampling periods of P = gens / (npass / ppp) generations, each run in ppp
// passes (the first ones one longer), so every sampled generation ends a
// pass: the last pass of each period.
__device__ __forceinline__ int pass_gens(const UnitRun &r, int pass) {
    if (r.ppp > 0) {
        const int P = r.gens / (r.npass / r.ppp), q = (pass - 1) % r.ppp;
        const int base = P / r.ppp, rem = P - base * r.ppp;
        return base + (q < rem ? 1 : 0);
    }
    const int base = r.gens / r.npass, rem = r.gens - base * r.npass;
    return base + (pass <= rem ? 1 : 0);
}

// Whole warp, after a pass that ends a sampling period of a population
// trace: the live cells of the words this warp stored in the pass (each
// lane reads back its own stores), reduced over the warp.  The units of a
// board cover its cells exactly once, so the board's count is the sum over
// its units.
__device__ __forceinline__ unsigned long long count_unit_output(const UnitRun &ud, const uint64_t *dst) {
    const int lane = threadIdx.x & 31;
    int seg = 0, word = 0;
    bool stores = false;
    if ((ud.mode & 0xff) == kUnitFull) {
        seg = lane / ud.W;
        word = lane - seg * ud.W;
        stores = seg < ud.S;
    } else {
        stores = lane >= 1 && lane <= ud.U;
        word = ud.w0 - 1 + lane;
        if (word >= ud.W) word -= ud.W;                 // tiles may wrap on a torus
    }
    unsigned long long c = 0;
    if (stores) {
        const int a = ud.r0 + seg * ud.H, e = min(a + ud.H, ud.r_end);
        const uint64_t *p = dst + word;
        for (int row = a; row < e; ++row) {
            const uint2 v = ld_cg_u64(p + (size_t)row * ud.W);
            c += __popc(v.x) + __popc(v.y);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    return c;
}

__device__ __forceinline__ int ld_relaxed(const int32_t *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int2 ld_relaxed_v2(const int32_t *p) {
    int2 v;
    asm volatile("ld.relaxed.gpu.global.v2.s32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void set_status(const PersistArgs &A, int code) {
    atomicCAS(&A.ctr[3], 0, code);
    atomicCAS(A.sticky, 0, code);
}

// Lane 0: wait until a queue slot that has been handed to this warp holds
// its unit (the filler took the slot from the ring's tail and is about to
// store it).  Returns the unit, or -1 if the launch failed or the wait gave up.
static __device__ int wait_slot(const PersistArgs &A, const int32_t *slot) {
    const uint64_t t0 = global_ns();
    unsigned ns = 32;
    for (long long spin = 0; spin < (1ll << 32); ++spin) {
        const int v = ld_acquire(slot);
        if (v >= 0) return v;
        if ((spin & 7) == 7) {
            if (ld_relaxed(&A.ctr[3]) != 0) return -1;
            if (global_ns() - t0 > (uint64_t)A.timeout_ns) {
                set_status(A, GOL_ETIMEOUT);
                return -1;
            }
        }
        __nanosleep(ns);
        if (ns < 128) ns <<= 1;
    }
    set_status(A, GOL_ETIMEOUT);
    return -1;
}

// Queues unit v for its next pass, rem = (npass - pass + 1) * cost being the
// rest of its chain: into the critical ring when rem >= hi_thr, else into
// the other one.  Each ring has a slot for every pass of its kind.
__device__ __forceinline__ void enqueue(const PersistArgs &A, int v, int64_t rem) {
    const bool hi = rem >= A.hi_thr;
    const int slot = atomicAdd(&A.qctr[hi ? 1 : 3], 1);
    const int64_t base = hi ? 0 : A.hi_cap, cap = hi ? A.hi_cap : A.total_tasks - A.hi_cap;
    if (slot < cap)
        st_release(&A.ring[base + slot], v);
    else
        set_status(A, GOL_ECUDA);              // the planner's ring sizes were wrong
}

// Lane 0: take the next pass to run.  A warp may hold one ticket of each
// ring (`tk[0]` critical, `tk[1]` other), taken with atomicAdd and kept until
// its slot is filled (or the launch ends), even while the warp runs other
// passes: a ticket is a promise to run what lands in its slot.  The warp
// takes a critical ticket when the critical ring shows queued passes (one
// load of its head and tail; the ticket may land past them and then waits
// for the next critical pass, alone for up to kCriticalWaitNs), otherwise an
// other-ring ticket, and serves whichever slot fills first, the critical one
// when both have.  Returns the
// unit (its pass is in next_pass), or -1 when every pass of the launch has
// completed or the launch failed.  Bounded: no completed pass for
// timeout_ns sets GOL_ETIMEOUT.
__device__ __forceinline__ int ticket_unit(const PersistArgs &A, int (&tk)[2]) {
    const int lo_cap = A.total_tasks - A.hi_cap;
    if (tk[0] >= 0 && tk[0] < A.hi_cap) {
        const int v = ld_acquire(&A.ring[tk[0]]);
        if (v >= 0) {
            tk[0] = -1;
            return v;
        }
    }
    if (tk[1] >= 0 && tk[1] < lo_cap) {
        const int v = ld_acquire(&A.ring[A.hi_cap + tk[1]]);
        if (v >= 0) {
            tk[1] = -1;
            return v;
        }
    }
    return -1;
}

// A critical ticket taken when the critical ring showed queued passes may
// land past them (other warps took those first).  Its holder waits up to
// kCriticalWaitNs for the next critical pass before it takes or serves
// other-ring work: a critical pass that lands in the slot of a warp busy
// with an other-ring pass waits for that pass to end (on the 4096-board
// batch the wait gains about 1 % of the makespan; windows of 20 to 200 us
// measure the same).  The wait is bounded: an endless one could leave every
// warp waiting for critical passes that are never queued.
constexpr uint64_t kCriticalWaitNs = 20000;

static __device__ int take_work(const PersistArgs &A, int (&tk)[2], uint32_t &tk0_ns) {
    uint64_t t_last = global_ns();
    int seen = -1;
    unsigned ns = 32;
    for (long long spin = 0; spin < (1ll << 32); ++spin) {
        // low 32 bits of the timer: the difference is exact for windows below 4 s
        const bool crit_wait = tk[0] >= 0 && tk[0] < A.hi_cap &&
                               (uint32_t)global_ns() - tk0_ns < (uint32_t)kCriticalWaitNs;
        if (crit_wait) {
            const int v = ld_acquire(&A.ring[tk[0]]);
            if (v >= 0) {
                tk[0] = -1;
                return v;
            }
        } else {
            const int v = ticket_unit(A, tk);
            if (v >= 0) return v;
        }
        if (tk[0] < 0 && A.hi_cap > 0 && (spin & 7) == 0) {
            const int2 ht = ld_relaxed_v2(&A.qctr[0]);
            if (ht.x < ht.y) {
                tk[0] = atomicAdd(&A.qctr[0], 1);
                tk0_ns = (uint32_t)global_ns();
                continue;
            }
        }
        if (tk[1] < 0 && !crit_wait) {
            tk[1] = atomicAdd(&A.qctr[2], 1);
            continue;
        }
        if ((spin & 7) == 7) {
            const int done = ld_relaxed(&A.ctr[2]);
            if (ld_relaxed(&A.ctr[3]) != 0 || done >= A.total_tasks) return -1;
            const uint64_t now = global_ns();
            if (done != seen) {
                seen = done;
                t_last = now;
            } else if (now - t_last > (uint64_t)A.timeout_ns) {
                set_status(A, GOL_ETIMEOUT);
                return -1;
            }
        }
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
    }
    set_status(A, GOL_ETIMEOUT);
    return -1;
}

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ void red_add(int32_t *p, int v) {
    asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int atom_add_acq_rel(int32_t *p, int v) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Whole warp, after unit u finished pass `pass`, with every lane's stores of
// the pass already ordered by an acquire-release fence and a warp barrier.
//
// Join counters: unit v may run pass q+1 once v and each of its nnb(v)
// neighbours have finished pass q.  join[v][q & 1] starts at nnb(v) + 1 and
// every finisher of pass q subtracts one for itself and for each of its
// neighbours (the relation is symmetric); the subtraction that reaches zero
// makes v ready, and only that one thread sees it, so v is claimed exactly
// once.  v restores the counter to nnb(v) + 1 when it starts pass q+1:
// nothing else touches that counter until v and its neighbours finish pass
// q+2, which needs v's pass q+1, so two parities suffice.  Lane 0 handles u
// itself and lane i its neighbour i - 1 (`my_nb`); the first ready lane's
// unit continues in this warp (at pass + 1, on the same board), the others
// are written their pass and go to the queue.  Returns the unit this warp
// runs next or -1.
__device__ __forceinline__ int complete_pass(const PersistArgs &A, int u, int pass, const UnitRun &r, int my_nb) {
    constexpr unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        red_add(&A.ctr[2], 1);
        if (pass == r.npass) {
            // last unit of the board to finish flips the board's current buffer
            if (atomicAdd(&A.ctr[4 + r.board], 1) == r.nunits - 1) {
                if (r.npass & 1) *r.curp ^= 1;
                A.ctr[4 + r.board] = 0;
            }
        }
    }
    if (pass >= r.npass) return -1;            // no unit of this board runs again
    if (r.nnb == 0) return u;                  // a board of one unit waits for nobody
    int v = -1;
    bool ready = false;
    if (lane <= r.nnb) {
        v = lane == 0 ? u : my_nb;
        ready = atom_add_acq_rel(&A.join[2 * v + (pass & 1)], -1) == 1;
    }
    const unsigned mask = __ballot_sync(kFull, ready);
    if (!mask) return -1;
    const int leader = __ffs(mask) - 1;
    const int next = __shfl_sync(kFull, v, leader);
    if (ready && lane != leader) {
        A.next_pass[v] = pass + 1;            // published by the queue slot's release
        enqueue(A, v, (int64_t)(r.npass - pass) * r.cost);
    }
    return next;
}

// Kernel variants: 0 window shift by register moves, 1 window slots rotated
// by renaming, 2 renaming with skewed stages, 3 = 1 held to three warps per
// scheduler at K = 8; 4, 5, 6 = 1 for boards with a masked last word (4),
// counting live cells for a population trace (5), or both (6), instantiated
// for K = 4, 6 and 8 only (kMaskedPopK).
constexpr bool variant_masked(int v) { return v == 4 || v == 6; }
constexpr bool variant_pop(int v) { return v == 5 || v == 6; }
constexpr bool variant_renaming(int v) { return v == 1 || v >= 3; }

// Blocks per SM the register allocation must allow (GOL_MIN_BLOCKS for
// K = 4..6 and GOL_MIN_BLOCKS_K8 for K = 8 at build time; 1 leaves the
// choice to the compiler).
#ifndef GOL_MIN_BLOCKS
#define GOL_MIN_BLOCKS 1
#endif
#ifndef GOL_MIN_BLOCKS_K8
#define GOL_MIN_BLOCKS_K8 1
#endif

// The skewed variant keeps K more register pairs; at K = 6 it is held to
// six blocks (three warps per scheduler) per SM.  Variant 3 is variant 1 held
// to six blocks per SM at K = 8 (168 registers instead of 185: three warps
// per scheduler instead of two), for launches with many units per warp.
template <int K, bool TORUS, int VARIANT>
__global__ void __launch_bounds__(kWarpsPerBlock * 32,
                                  (K >= 4 && K <= 6) ? (VARIANT == 2 && GOL_MIN_BLOCKS < 6 ? 6 : GOL_MIN_BLOCKS)
                                                     : (K == 8 ? (VARIANT == 3 ? 6 : GOL_MIN_BLOCKS_K8) : 1))
persistent_step_kernel(const PersistArgs A) {
    constexpr unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * kWarpsPerBlock + (int)(threadIdx.x >> 5);
    // warp w < hi_init starts with the critical ring's slot w (pass 1)
    int u = w < min(A.hi_init, A.nwarps) ? A.ring[w] : -1, pass = 1;
    // lane 0's scheduling state, in shared memory (used between passes only,
    // it stays out of the registers of the pass): the tickets this warp holds
    // (critical, other) and when it took its critical ticket
    __shared__ int s_tk[kWarpsPerBlock][2];
    __shared__ uint32_t s_tk0[kWarpsPerBlock];
    int (&tk)[2] = s_tk[threadIdx.x >> 5];
    uint32_t &tk0_ns = s_tk0[threadIdx.x >> 5];
    if (lane == 0) {
        tk[0] = tk[1] = -1;
        tk0_ns = 0;
    }
    for (;;) {
        if (u < 0) {
            int v = -1, p = 0;
            if (lane == 0) {
                v = take_work(A, tk, tk0_ns);
                // written before the slot by the thread that queued v; the
                // slot's acquire load orders this read after it
                if (v >= 0) p = A.next_pass[v];
            }
            u = __shfl_sync(kFull, v, 0);
            if (u < 0) return;
            pass = __shfl_sync(kFull, p, 0);
        }
        const UnitRun r = A.run[u];
        const int my_nb = (lane >= 1 && lane <= kMaxNeighbours) ? A.run[u].nb[lane - 1] : u;
        // restore the join counter that made u ready (see complete_pass)
        if (lane == 0 && pass > 1) A.join[2 * u + ((pass - 1) & 1)] = r.nnb + 1;
        const uint64_t *src = r.buf[(r.cur + pass - 1) & 1];
        uint64_t *dst = r.buf[(r.cur + pass) & 1];
        const int kk = pass_gens(r, pass);
        constexpr bool MASKED = variant_masked(VARIANT);
        if (VARIANT == 0) {
            if (kk == K)
                run_unit_pass_moves<K, TORUS, false>(r, src, dst, K);
            else
                run_unit_pass_moves<K, TORUS, true>(r, src, dst, kk);
        } else if (variant_renaming(VARIANT)) {
            if (kk == K)
                run_unit_pass<K, TORUS, false, MASKED>(r, src, dst, K);
            else
                run_unit_pass<K, TORUS, true, MASKED>(r, src, dst, kk);
        } else {
            if (kk == K)
                run_unit_pass_skew<K, TORUS, false>(r, src, dst, K);
            else
                run_unit_pass_skew<K, TORUS, true>(r, src, dst, kk);
        }
        if (variant_pop(VARIANT) && r.ppp > 0 && pass % r.ppp == 0) {
            const unsigned long long c = count_unit_output(r, dst);
            if (lane == 0) atomicAdd(&A.pop[r.pop_off + pass / r.ppp - 1], c);
        }
        // every lane's stores of this pass (and the counter reset) are ordered
        // before the counter updates that publish it (acquire-release fence,
        // then the warp barrier)
        fence_acq_rel_gpu();
        __syncwarp();
        const int next = complete_pass(A, u, pass, r, my_nb);
        // a filled ticket runs before a continuation in this warp, which is
        // queued instead (so that no ticket waits on a chain)
        int take = -1, tpass = 0;
        if (lane == 0 && next >= 0 && (tk[0] >= 0 || tk[1] >= 0)) {
            const int v = ticket_unit(A, tk);
            if (v >= 0) {
                A.next_pass[next] = pass + 1;
                enqueue(A, next, (int64_t)(r.npass - pass) * r.cost);
                take = v;
                tpass = A.next_pass[v];
            }
        }
        take = __shfl_sync(kFull, take, 0);
        if (take >= 0) {
            u = take;
            pass = __shfl_sync(kFull, tpass, 0);
        } else if (next >= 0) {
            u = next;
            ++pass;          // continuing in this warp: the next pass of a unit of the same board
        } else {
            u = -1;
        }
    }
}

template <int K, int V>
cudaError_t launch_variant(const PersistArgs &a, bool torus, int grid, cudaStream_t s) {
    if (torus)
        persistent_step_kernel<K, true, V><<<grid, kWarpsPerBlock * 32, 0, s>>>(a);
    else
        persistent_step_kernel<K, false, V><<<grid, kWarpsPerBlock * 32, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

template <int K, int V>
cudaError_t occupancy_variant(bool torus, int *bps) {
    const int t = kWarpsPerBlock * 32;
    return torus ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, persistent_step_kernel<K, true, V>, t, 0)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, persistent_step_kernel<K, false, V>, t, 0);
}

// generations per pass with instantiations of variants 4, 5 and 6
constexpr bool masked_pop_k(int k) { return k == 4 || k == 6 || k == 8; }

template <int K>
cudaError_t launch_persistent_impl(const PersistArgs &a, bool torus, int variant, int grid, cudaStream_t s) {
    if constexpr (masked_pop_k(K)) {
        if (variant == 4) return launch_variant<K, 4>(a, torus, grid, s);
        if (variant == 5) return launch_variant<K, 5>(a, torus, grid, s);
        if (variant == 6) return launch_variant<K, 6>(a, torus, grid, s);
    }
    if (variant >= 4) return cudaErrorInvalidValue;
    if (variant == 0) return launch_variant<K, 0>(a, torus, grid, s);
    if (variant == 2) return launch_variant<K, 2>(a, torus, grid, s);
    if (variant == 3 && K == 8) return launch_variant<K, (K == 8 ? 3 : 1)>(a, torus, grid, s);
    return launch_variant<K, 1>(a, torus, grid, s);
}

template <int K>
cudaError_t persistent_occupancy_impl(bool torus, int variant, int *bps) {
    if constexpr (masked_pop_k(K)) {
        if (variant == 4) return occupancy_variant<K, 4>(torus, bps);
        if (variant == 5) return occupancy_variant<K, 5>(torus, bps);
        if (variant == 6) return occupancy_variant<K, 6>(torus, bps);
    }
    if (variant >= 4) return cudaErrorInvalidValue;
    if (variant == 0) return occupancy_variant<K, 0>(torus, bps);
    if (variant == 2) return occupancy_variant<K, 2>(torus, bps);
    if (variant == 3 && K == 8) return occupancy_variant<K, (K == 8 ? 3 : 1)>(torus, bps);
    return occupancy_variant<K, 1>(torus, bps);
}

#define GOL_INSTANTIATE_PERSISTENT(KV)                                                             \
    template <>                                                                                    \
    cudaError_t launch_persistent<KV>(const PersistArgs &a, bool torus, int variant, int grid,     \
                                      cudaStream_t s) {                                            \
        return launch_persistent_impl<KV>(a, torus, variant, grid, s);                             \
    }                                                                                              \
    template <>                                                                                    \
    cudaError_t persistent_occupancy<KV>(bool torus, int variant, int *bps) {                      \
        return persistent_occupancy_impl<KV>(torus, variant, bps);                                 \
    }

}  // namespace gol
