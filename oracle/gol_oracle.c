/*
 * Oracle for the Game of Life generation step: a plain, serial, one-byte-
 * per-cell CPU implementation written straight from the paper's statement
 * of the problem.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load it.  It shares no code, header or table
 * with the CUDA path.
 *
 * What it computes (Section 1 of the paper, and Section 2.2 for the edges):
 *
 *   n(r,c)  = sum over the eight offsets (dr,dc) in {-1,0,1}^2 \ {(0,0)} of
 *             X[(r+dr) mod R][(c+dc) mod C]             (torus, Section 2.2)
 *             or of X at (r+dr, c+dc) with cells outside the board dead
 *             (bounded board, "torus = 0")
 *   X'(r,c) = the four transitions of Section 1, written case by case in
 *             transition() below.
 *
 * Readings taken where the paper is silent:
 *   - a dead cell with a neighbour count other than three stays dead (the
 *     four listed transitions do not cover it);
 *   - all cells change at once, each from the previous generation only
 *     ("at each step in time"), so two buffers are used;
 *   - on tori with fewer than three rows or columns the wrapped offsets
 *     name the same cell more than once and it is counted once per offset,
 *     exactly as the sum above says.
 *
 * Cells are uint8 0/1, row major, R rows of C columns.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)

/* State of cell (r, c); (r, c) may lie outside [0,R) x [0,C). */
static int cell_at(const uint8_t *X, int64_t R, int64_t C, int torus,
                   int64_t r, int64_t c)
{
    if (torus) {
        r = ((r % R) + R) % R; /* left/right and top/bottom edges adjacent */
        c = ((c % C) + C) % C;
    } else if (r < 0 || r >= R || c < 0 || c >= C) {
        return 0;
    }
    return X[r * C + c] ? 1 : 0;
}

/* The eight neighbours: horizontally, vertically or diagonally adjacent. */
static int neighbour_count(const uint8_t *X, int64_t R, int64_t C, int torus,
                           int64_t r, int64_t c)
{
    int n = 0;
    for (int dr = -1; dr <= 1; ++dr)
        for (int dc = -1; dc <= 1; ++dc)
            if (dr != 0 || dc != 0)
                n += cell_at(X, R, C, torus, r + dr, c + dc);
    return n;
}

/* The transitions of Section 1, in the paper's order. */
static uint8_t transition(int alive, int n)
{
    if (alive) {
        if (n < 2)
            return 0; /* 1: fewer than two live neighbours, dies           */
        if (n == 2 || n == 3)
            return 1; /* 2: two or three live neighbours, lives on          */
        return 0;     /* 3: more than three live neighbours, dies           */
    }
    if (n == 3)
        return 1;     /* 4: dead with exactly three live neighbours, born   */
    return 0;         /* not named by the paper: a dead cell stays dead     */
}

static int check_args(int64_t R, int64_t C, const void *in, const void *out)
{
    if (R < 0 || C < 0)
        return ORACLE_EINVAL;
    if (R > 0 && C > 0 && (!in || !out))
        return ORACLE_EINVAL;
    return ORACLE_OK;
}

/* One generation, serial.  in and out must not overlap. */
int oracle_step(int64_t R, int64_t C, int torus, const uint8_t *in, uint8_t *out)
{
    int rc = check_args(R, C, in, out);
    if (rc)
        return rc;
    for (int64_t r = 0; r < R; ++r)
        for (int64_t c = 0; c < C; ++c)
            out[r * C + c] = transition(in[r * C + c] != 0,
                                        neighbour_count(in, R, C, torus, r, c));
    return ORACLE_OK;
}

/* G generations, serial; in and out may be the same buffer. */
int oracle_run(int64_t R, int64_t C, int torus, int64_t G,
               const uint8_t *in, uint8_t *out)
{
    int rc = check_args(R, C, in, out);
    if (rc || G < 0)
        return rc ? rc : ORACLE_EINVAL;
    size_t n = (size_t)R * (size_t)C;
    if (n == 0)
        return ORACLE_OK;
    uint8_t *a = (uint8_t *)malloc(n), *b = (uint8_t *)malloc(n);
    if (!a || !b) {
        free(a);
        free(b);
        return ORACLE_ENOMEM;
    }
    memcpy(a, in, n);
    for (int64_t g = 0; g < G; ++g) {
        oracle_step(R, C, torus, a, b);
        uint8_t *t = a;
        a = b;
        b = t;
    }
    memcpy(out, a, n);
    free(a);
    free(b);
    return ORACLE_OK;
}

/* ---------------------------------------------------------------------------
 * The paper's domain decompositions (Section 2.1 and 2.2) as OpenMP
 * programs.  Each thread owns one part of the board and computes it with
 * the same per-cell arithmetic as oracle_step.  They exist as timed CPU
 * baselines and as a check that a decomposition never changes the result.
 * ------------------------------------------------------------------------- */

static void step_rect(int64_t R, int64_t C, int torus, const uint8_t *in,
                      uint8_t *out, int64_t r0, int64_t r1, int64_t c0, int64_t c1)
{
    for (int64_t r = r0; r < r1; ++r)
        for (int64_t c = c0; c < c1; ++c)
            out[r * C + c] = transition(in[r * C + c] != 0,
                                        neighbour_count(in, R, C, torus, r, c));
}

/* parts x parts_c decomposition: mode 0 = bars of rows, 1 = bars of
 * columns, 2 = an m x n grid of blocks (m = parts, n = parts_c). */
static int run_decomposed(int mode, int64_t R, int64_t C, int torus, int64_t G,
                          const uint8_t *in, uint8_t *out, int threads,
                          int parts_c)
{
    int rc = check_args(R, C, in, out);
    if (rc || G < 0 || threads < 1 || (mode == 2 && parts_c < 1))
        return rc ? rc : ORACLE_EINVAL;
    size_t n = (size_t)R * (size_t)C;
    if (n == 0)
        return ORACLE_OK;
    uint8_t *a = (uint8_t *)malloc(n), *b = (uint8_t *)malloc(n);
    if (!a || !b) {
        free(a);
        free(b);
        return ORACLE_ENOMEM;
    }
    memcpy(a, in, n);
    int parts_r = threads;
    int nparts = mode == 2 ? parts_r * parts_c : threads;
    int nthreads = nparts;
    for (int64_t g = 0; g < G; ++g) {
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static)
#endif
        for (int p = 0; p < nparts; ++p) {
            int64_t r0 = 0, r1 = R, c0 = 0, c1 = C;
            if (mode == 0) {
                r0 = R * p / nparts;
                r1 = R * (p + 1) / nparts;
            } else if (mode == 1) {
                c0 = C * p / nparts;
                c1 = C * (p + 1) / nparts;
            } else {
                int pr = p / parts_c, pc = p % parts_c;
                r0 = R * pr / parts_r;
                r1 = R * (pr + 1) / parts_r;
                c0 = C * pc / parts_c;
                c1 = C * (pc + 1) / parts_c;
            }
            step_rect(R, C, torus, a, b, r0, r1, c0, c1);
        }
        uint8_t *t = a;
        a = b;
        b = t;
    }
    memcpy(out, a, n);
    free(a);
    free(b);
    return ORACLE_OK;
}

/* Section 2.1, by rows: each of `threads` threads owns a bar of rows. */
int oracle_run_rows_omp(int64_t R, int64_t C, int torus, int64_t G,
                        const uint8_t *in, uint8_t *out, int threads)
{
    return run_decomposed(0, R, C, torus, G, in, out, threads, 1);
}

/* Section 2.1, by columns: each thread owns a bar of columns. */
int oracle_run_cols_omp(int64_t R, int64_t C, int torus, int64_t G,
                        const uint8_t *in, uint8_t *out, int threads)
{
    return run_decomposed(1, R, C, torus, G, in, out, threads, 1);
}

/* Section 2.2: an m x n grid of equal blocks, run on m*n threads. */
int oracle_run_blocks_omp(int64_t R, int64_t C, int torus, int64_t G,
                          const uint8_t *in, uint8_t *out, int m, int n)
{
    if (m < 1 || n < 1)
        return ORACLE_EINVAL;
    return run_decomposed(2, R, C, torus, G, in, out, m, n);
}

/* Table 1's quantity: the number of live cells. */
int oracle_population(int64_t R, int64_t C, const uint8_t *cells, uint64_t *out)
{
    if (R < 0 || C < 0 || !out || (R > 0 && C > 0 && !cells))
        return ORACLE_EINVAL;
    uint64_t s = 0;
    for (int64_t i = 0; i < R * C; ++i)
        s += cells[i] ? 1u : 0u;
    *out = s;
    return ORACLE_OK;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
