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
