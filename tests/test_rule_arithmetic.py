"""The kernels' rule arithmetic, checked on the CPU from the CUDA source.

The packed kernel evaluates the four transitions of Section 1 bit-sliced:
three-cell row sums as two bit planes, then a straight-line program of
3-input LOP3 operations (`rule32` in wavefront.cuh); the cluster-resident
byte kernel writes the same predicate with C operators (`byte_rule` in
kernels_util.cu).  These tests read those functions out of the source,
interpret them on single bits, and compare them with B3/S23 on all 512 3x3
neighbourhoods, so a wrong LUT immediate or operand order fails here
without a GPU.  (The GPU parity tests check the compiled kernels.)
"""
import itertools
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1209_4408_gb300", "csrc")


def source(name):
    with open(os.path.join(CSRC, name)) as f:
        return f.read()


def function_body(text, name):
    m = re.search(r"\b%s\s*\(" % re.escape(name), text)
    assert m, name
    i = text.index("{", m.end())
    depth, j = 0, i
    while True:
        if text[j] == "{":
            depth += 1
        elif text[j] == "}":
            depth -= 1
            if depth == 0:
                return text[i + 1:j]
        j += 1


def lop3(lut, a, b, c):
    """PTX lop3.b32 on single bits: bit (4a + 2b + c) of the LUT, with the
    operand constants a = 0xF0, b = 0xCC, c = 0xAA."""
    return (lut >> (4 * a + 2 * b + c)) & 1


def lut_constants(text):
    return {m.group(1): int(m.group(2), 0)
            for m in re.finditer(r"constexpr\s+unsigned\s+(\w+)\s*=\s*(0x[0-9A-Fa-f]+|\d+)\s*;", text)}


def rule32_program():
    text = source("wavefront.cuh")
    consts = lut_constants(text)
    body = function_body(text, "rule32")
    steps = []
    for m in re.finditer(r"(?:const\s+uint32_t\s+(\w+)\s*=|return)\s*lop3<(\w+)>\((\w+),\s*(\w+),\s*(\w+)\)\s*;", body):
        dst, lut, a, b, c = m.groups()
        lut = consts[lut] if lut in consts else int(lut, 0)
        steps.append((dst or "return", lut, a, b, c))
    assert steps and steps[-1][0] == "return"
    return steps


def run_rule32(steps, t0, t1, m0, m1, b0, b1, a):
    env = dict(t0=t0, t1=t1, m0=m0, m1=m1, b0=b0, b1=b1, a=a)
    for dst, lut, x, y, z in steps:
        env[dst] = lop3(lut, env[x], env[y], env[z])
    return env["return"]


def byte_rule_eval():
    body = function_body(source("kernels_util.cu"), "byte_rule")
    body = re.sub(r"//[^\n]*", "", body)
    decls, ret = [], None
    for stmt in body.split(";"):
        stmt = stmt.strip()
        if stmt.startswith("const uint64_t"):
            decls.extend(d.strip() for d in stmt[len("const uint64_t"):].split(","))
        elif stmt.startswith("return"):
            ret = stmt[len("return"):].strip()

    # only names, bitwise operators and parentheses are evaluated
    for e in [d.split("=", 1)[1] for d in decls] + [ret]:
        assert re.fullmatch(r"[\w\s^&|~()]+", e), e

    def f(t0, t1, m0, m1, b0, b1, a):
        env = dict(t0=t0, t1=t1, m0=m0, m1=m1, b0=b0, b1=b1, a=a)
        for d in decls:
            name, expr = d.split("=", 1)
            env[name.strip()] = eval(expr, {}, env) & 1
        return eval(ret, {}, env) & 1
    return f


def b3s23(block):
    alive = block[1][1]
    n = sum(block[r][c] for r in range(3) for c in range(3)) - alive
    return 1 if n == 3 or (alive and n == 2) else 0


def planes(row):
    s = sum(row)                    # west + cell + east
    return s & 1, s >> 1


def test_lop3_luts_name_their_functions():
    consts = lut_constants(source("wavefront.cuh"))
    for a, b, c in itertools.product((0, 1), repeat=3):
        assert lop3(consts["kXor3"], a, b, c) == a ^ b ^ c
        assert lop3(consts["kMaj3"], a, b, c) == (a + b + c >= 2)
    # the operand convention itself: f(0xF0, 0xCC, 0xAA) is the LUT
    for lut in (0x96, 0xE8, 0x14, 0x82, 0x60, 0xCA):
        assert sum(lop3(lut, (0xF0 >> i) & 1, (0xCC >> i) & 1, (0xAA >> i) & 1) << i for i in range(8)) == lut


def test_rule32_on_all_512_neighbourhoods():
    steps = rule32_program()
    assert len(steps) == 8          # eight LOP3 per 32-bit half, as the operation count states
    for bits in range(512):
        block = [[(bits >> (3 * r + c)) & 1 for c in range(3)] for r in range(3)]
        (t0, t1), (m0, m1), (b0, b1) = (planes(r) for r in block)
        got = run_rule32(steps, t0, t1, m0, m1, b0, b1, block[1][1])
        assert got == b3s23(block), (bits, block)


def test_byte_rule_on_all_512_neighbourhoods():
    f = byte_rule_eval()
    for bits in range(512):
        block = [[(bits >> (3 * r + c)) & 1 for c in range(3)] for r in range(3)]
        (t0, t1), (m0, m1), (b0, b1) = (planes(r) for r in block)
        assert f(t0, t1, m0, m1, b0, b1, block[1][1]) == b3s23(block), (bits, block)


def test_a_wrong_lut_is_caught():
    """The check is sharp: flipping one bit of one LUT of rule32 breaks some
    neighbourhood in all but a few cases (LUT entries that no valid input
    selects, or whose effect a later operation masks)."""
    steps = rule32_program()
    cases = []
    for bits in range(512):
        block = [[(bits >> (3 * r + c)) & 1 for c in range(3)] for r in range(3)]
        (t0, t1), (m0, m1), (b0, b1) = (planes(r) for r in block)
        cases.append(((t0, t1, m0, m1, b0, b1, block[1][1]), b3s23(block)))
    caught = total = 0
    for k in range(len(steps)):
        for bit in range(8):
            mutated = list(steps)
            dst, lut, a, b, c = mutated[k]
            mutated[k] = (dst, lut ^ (1 << bit), a, b, c)
            total += 1
            caught += any(run_rule32(mutated, *args) != want for args, want in cases)
    assert caught >= 0.9 * total, (caught, total)


# ---------------------------------------------------------------------------
# Row sums of the packed kernel (even/odd split words, funnel shifts, lane
# shuffles), read from each pass variant of wavefront.cuh.
# ---------------------------------------------------------------------------
M32 = 0xFFFFFFFF


def lop3_words(lut, a, b, c):
    """lop3.b32 on numpy uint32 arrays (the sum of the LUT's minterms)."""
    import numpy as np

    out = np.zeros_like(a)
    for idx in range(8):
        if (lut >> idx) & 1:
            out |= (a if idx & 4 else ~a) & (b if idx & 2 else ~b) & (c if idx & 1 else ~c)
    return out


def funnelshift(kind, lo, hi, n):
    """CUDA __funnelshift_l / __funnelshift_r: the high (l) or low (r) 32 bits
    of the 64-bit value hi:lo shifted left / right by n & 31; "rc" is
    __funnelshift_rc, the right shift by min(n, 32)."""
    import numpy as np

    v = (hi.astype(np.uint64) << np.uint64(32)) | lo.astype(np.uint64)
    if kind == "rc":
        return (v >> np.uint64(min(n, 32))).astype(np.uint32)
    n = np.uint64(n & 31)
    if kind == "l":
        return ((v << n) >> np.uint64(32)).astype(np.uint32)
    return (v >> n).astype(np.uint32)


def braced(text, start):
    """The text inside the first {...} block at or after `start`."""
    i = text.index("{", start)
    depth = 0
    for j in range(i, len(text)):
        depth += {"{": 1, "}": -1}.get(text[j], 0)
        if depth == 0:
            return text[i + 1:j]
    raise AssertionError("unbalanced braces")


def iterate_bodies():
    """Bodies of the `iterate` lambdas (one per pass variant)."""
    text = source("wavefront.cuh")
    return [braced(text, m.end()) for m in re.finditer(r"auto iterate = \[&\]\([^)]*\)", text)]


def row_sum_program(body):
    consts = lut_constants(source("wavefront.cuh"))
    shifts = {m.group(1): (m.group(2), m.group(3), m.group(4), int(m.group(5)))
              for m in re.finditer(r"(\w+) = __funnelshift_([lr])\((\w+),\s*(\w+),\s*(\d+)\)", body)}
    planes = []
    for m in re.finditer(r"(\w+)(?:\[\w+\])*\s*=\s*lop3<(\w+)>\((\w+),\s*(\w+),\s*(\w+)\)", body):
        name, lut, a, b, c = m.groups()
        if name in ("xl", "xh"):
            continue                    # the masked last word's padding patch (see masked_program)
        pm = re.fullmatch(r"[a-z]([01])([lh])", name)
        assert pm, name
        planes.append((int(pm.group(1)), pm.group(2), consts.get(lut, None) or int(lut, 0), a, b, c))
    return shifts, planes


def to_halves(cells_row):
    """A row of 64 W cells in the resident layout: per word, the low half
    holds the even columns (bit j = column 2j), the high half the odd ones."""
    import numpy as np

    w = cells_row.reshape(-1, 64).astype(np.uint64)
    j = np.arange(32, dtype=np.uint64)
    lo = (w[:, 0::2] << j).sum(axis=1).astype(np.uint32)
    hi = (w[:, 1::2] << j).sum(axis=1).astype(np.uint32)
    return lo, hi


def from_halves(lo, hi):
    import numpy as np

    j = np.arange(32, dtype=np.uint32)
    cells = np.zeros((lo.size, 64), np.uint8)
    cells[:, 0::2] = (lo[:, None] >> j) & 1
    cells[:, 1::2] = (hi[:, None] >> j) & 1
    return cells.reshape(-1)


def kernel_planes(shifts, planes, lo, hi):
    """Row-sum planes of one row of a torus held as one segment of W lanes:
    lane k holds word k; the west / east lanes are k -+ 1 mod W."""
    import numpy as np

    env = {"xl": lo, "xh": hi, "wh": np.roll(hi, 1), "el": np.roll(lo, -1)}
    for dst, (kind, a, b, n) in shifts.items():
        env[dst] = funnelshift(kind, env[a], env[b], n)
    out = {}
    for plane, half, lut, a, b, c in planes:
        out[(plane, half)] = lop3_words(lut, env[a], env[b], env[c])
    return out


def test_row_sums_of_every_pass_variant():
    import numpy as np

    bodies = iterate_bodies()
    assert len(bodies) == 3                      # register moves, renaming, skewed stages
    rng = np.random.default_rng(44)
    for body in bodies:
        shifts, planes = row_sum_program(body)
        assert sorted((p, h) for p, h, *_ in planes) == [(0, "h"), (0, "l"), (1, "h"), (1, "l")]
        for W in (1, 2, 3, 5):
            row = (rng.random(64 * W) < 0.5).astype(np.uint8)
            got = kernel_planes(shifts, planes, *to_halves(row))
            hsum = np.roll(row, 1) + row + np.roll(row, -1)          # west + cell + east on the torus
            for plane in (0, 1):
                want = (hsum >> plane) & 1
                assert np.array_equal(from_halves(got[(plane, "l")], got[(plane, "h")]), want), (plane, W)


def test_rule_call_takes_the_middle_row_alive_word():
    """rule32(t0, t1, m0, m1, b0, b1, alive): the alive word comes from the
    same window slot as the middle row's planes, the three rows' planes from
    three different slots, and each call reads one half only."""
    for body in iterate_bodies():
        calls = re.findall(r"rule32\(([^;]*)\)\s*;", body)
        assert len(calls) == 2, calls
        for call in calls:
            args = [a.strip() for a in call.split(",")]
            assert len(args) == 7

            def slot(x):
                return (x[0], x[x.index("["):] if "[" in x else "")

            assert slot(args[0]) == slot(args[1]) and slot(args[4]) == slot(args[5])
            assert slot(args[2]) == slot(args[3]) == slot(args[6])
            assert len({slot(args[0]), slot(args[2]), slot(args[4])}) == 3
            halves = {a.split("[")[0][-1] for a in args}
            assert len(halves) == 1 and halves <= {"l", "h"}, args


def test_one_generation_from_the_kernel_source_matches_the_oracle():
    """Row sums (parsed) + rule32 (parsed), composed over rows above, at and
    below on a torus, equal the oracle's generation."""
    import numpy as np

    oracle = __import__("pytest").importorskip("oracle")
    steps = rule32_program()
    shifts, planes = row_sum_program(iterate_bodies()[1])
    rng = np.random.default_rng(45)

    def rule_words(t, m, b, alive):
        out = np.zeros_like(alive)
        for bit in range(32):
            sel = np.uint32(1 << bit)
            for i in range(alive.size):
                args = [int((x[i] & sel) != 0) for x in (t[0], t[1], m[0], m[1], b[0], b[1], alive)]
                if run_rule32(steps, *args):
                    out[i] |= sel
        return out

    for R, W in ((3, 1), (5, 2), (4, 3)):
        cells = (rng.random((R, 64 * W)) < 0.4).astype(np.uint8)
        halves = [to_halves(cells[r]) for r in range(R)]
        pl = [kernel_planes(shifts, planes, lo, hi) for lo, hi in halves]
        nxt = np.zeros_like(cells)
        for r in range(R):
            above, mid, below = pl[(r - 1) % R], pl[r], pl[(r + 1) % R]
            lo = rule_words((above[(0, "l")], above[(1, "l")]), (mid[(0, "l")], mid[(1, "l")]),
                            (below[(0, "l")], below[(1, "l")]), halves[r][0])
            hi = rule_words((above[(0, "h")], above[(1, "h")]), (mid[(0, "h")], mid[(1, "h")]),
                            (below[(0, "h")], below[(1, "h")]), halves[r][1])
            nxt[r] = from_halves(lo, hi)
        assert np.array_equal(nxt, oracle.run(cells, 1)), (R, W)


# ---------------------------------------------------------------------------
# Boards whose width is not a multiple of 64: the masked stage arithmetic of
# the renaming pass variant (the padding patch of the last word and the value
# sent west to word 0), read from the source and run on rows of every width.
# ---------------------------------------------------------------------------
def masked_program(body):
    """(wsend LUT, patch LUTs) of the MASKED lines of an iterate body."""
    consts = lut_constants(source("wavefront.cuh"))
    m = re.search(r"wsend = __funnelshift_rc\(xh, lop3<(\w+)>\(xh, xl, west_pick\), west_n\);", body)
    assert m, "west value of the masked last word"
    wlut = consts.get(m.group(1), None) or int(m.group(1), 0)
    m = re.search(r"const uint32_t t = el << pad_shift;", body)
    assert m, "padding bit shift"
    pl = re.search(r"xl = lop3<(\w+)>\(xl, t, pad_l\);", body)
    ph = re.search(r"xh = lop3<(\w+)>\(xh, t, pad_h\);", body)
    assert pl and ph, "padding patches"
    return wlut, int(pl.group(1), 0), int(ph.group(1), 0)


def last_lane_constants(cl):
    """The masked last word's lane constants as the kernel documents them:
    column 0 goes to the first padding column (even C': low half bit C'/2,
    odd C': high half bit (C'-1)/2); bit 31 of the value sent west is column
    C - 1 (even C': high half bit C'/2 - 1, odd C': low half bit (C'-1)/2)."""
    shift = cl >> 1
    pad_l = 0 if cl & 1 else 1 << shift
    pad_h = 1 << shift if cl & 1 else 0
    return shift, pad_l, pad_h, (cl + 1) >> 1, (M32 if cl & 1 else 0)


def test_masked_last_word_row_sums_every_width():
    import numpy as np

    bodies = iterate_bodies()
    body = bodies[1]                                 # the renaming variant carries the masked path
    wlut, plut, hlut = masked_program(body)
    shifts, planes = row_sum_program(body)
    rng = np.random.default_rng(46)
    for C in list(range(1, 130)) + [191, 200]:
        if C % 64 == 0:
            continue
        W, cl = (C + 63) // 64, C % 64
        for trial in range(3):
            row = (rng.random(C) < 0.5).astype(np.uint8)
            padded = np.zeros(64 * W, np.uint8)
            padded[:C] = row
            lo, hi = to_halves(padded)
            # padding of words that have left a stage is arbitrary: garbage
            garbage = rng.integers(0, 1 << 32, size=2, dtype=np.uint64).astype(np.uint32)
            keep_l = M32 if (cl + 1) >> 1 >= 32 else (1 << ((cl + 1) >> 1)) - 1
            keep_h = (1 << (cl >> 1)) - 1
            lo[-1] = (lo[-1] & np.uint32(keep_l)) | (garbage[0] & np.uint32(~keep_l & M32))
            hi[-1] = (hi[-1] & np.uint32(keep_h)) | (garbage[1] & np.uint32(~keep_h & M32))
            shift, pad_l, pad_h, west_n, pick = last_lane_constants(cl)
            z = np.zeros(W, np.uint32)
            sh, pl_, ph_, wn, pk = z.copy(), z.copy(), z.copy(), np.zeros(W, np.int64), z.copy()
            sh[-1], pl_[-1], ph_[-1], wn[-1], pk[-1] = shift, pad_l, pad_h, west_n, pick
            wsend = np.array([funnelshift("rc", hi[k:k + 1], lop3_words(wlut, hi[k:k + 1], lo[k:k + 1], pk[k:k + 1]),
                                          int(wn[k]))[0] for k in range(W)], dtype=np.uint32)
            wh, el = np.roll(wsend, 1), np.roll(lo, -1)
            t = (el.astype(np.uint64) << sh.astype(np.uint64)).astype(np.uint64) & np.uint64(M32)
            t = t.astype(np.uint32)
            lo2, hi2 = lop3_words(plut, lo, t, pl_), lop3_words(hlut, hi, t, ph_)
            env = {"xl": lo2, "xh": hi2, "wh": wh, "el": el}
            for dst, (kind, a, b, n) in shifts.items():
                env[dst] = funnelshift(kind, env[a], env[b], n)
            got = {}
            for plane, half, lut, a, b, c in planes:
                got[(plane, half)] = lop3_words(lut, env[a], env[b], env[c])
            hsum = np.roll(row, 1) + row + np.roll(row, -1)          # the C-column torus
            for plane in (0, 1):
                cells = from_halves(got[(plane, "l")], got[(plane, "h")])[:C]
                assert np.array_equal(cells, (hsum >> plane) & 1), (C, plane)
