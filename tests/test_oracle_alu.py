"""Pins the oracle's ALU/JMP semantics by brute force against an independent big-int model.

Every operation of RFC 9669 Sec. 4.1-4.3 is run through the C oracle over a table of
edge-case operands (0, +-1, INT32/INT64 limits, 2^32, all-ones, shift counts 63/64/65, ...)
in both register (X) and immediate (K) forms and both widths, and compared with
`ebpf_model`, which is written separately in Python.
"""
import itertools

import numpy as np
import pytest

import oracle as O
from tests import ebpf_model as M
from workloads.asm import Asm

OPS = ["add", "sub", "mul", "div", "mod", "or", "and", "xor", "lsh", "rsh", "arsh", "mov"]
PAIRS = list(itertools.product(M.INTERESTING, M.INTERESTING))


def ctx_pairs(pairs):
    arr = np.zeros((len(pairs), 2), dtype=np.uint64)
    for i, (a, b) in enumerate(pairs):
        arr[i, 0], arr[i, 1] = a, b
    return arr


def run_r0(a: Asm, ctx: np.ndarray) -> np.ndarray:
    r0, _ = O.run(a.prog(), [], ctx, 16, want_r0=True)
    return r0.view(np.uint64)


@pytest.mark.parametrize("bits", [64, 32])
@pytest.mark.parametrize("op", OPS + ["sdiv", "smod"])
def test_alu_reg_form(op, bits):
    off = 1 if op in ("sdiv", "smod") else 0
    base = {"sdiv": "div", "smod": "mod"}.get(op, op)
    a = Asm().ldx(8, "r0", "r1", 0).ldx(8, "r2", "r1", 8).alu(base, "r0", "r2", bits=bits, off=off).exit()
    got = run_r0(a, ctx_pairs(PAIRS))
    want = [M.alu(base, bits, d, s, off) for d, s in PAIRS]
    bad = [(hex(d), hex(s), hex(int(g)), hex(w)) for (d, s), g, w in zip(PAIRS, got, want) if int(g) != w]
    assert not bad, bad[:5]


@pytest.mark.parametrize("bits", [64, 32])
@pytest.mark.parametrize("op", OPS + ["sdiv", "smod"])
def test_alu_imm_form(op, bits):
    off = 1 if op in ("sdiv", "smod") else 0
    base = {"sdiv": "div", "smod": "mod"}.get(op, op)
    ds = M.INTERESTING
    ctx = ctx_pairs([(d, 0) for d in ds])
    for imm in M.INTERESTING_IMM:
        a = Asm().ldx(8, "r0", "r1", 0).alu(base, "r0", imm, bits=bits, off=off).exit()
        got = run_r0(a, ctx)
        # the immediate is sign-extended to 64 bits for ALU64 and used as 32 bits for ALU
        s = imm & M.mask(64) if bits == 64 else imm & M.mask(32)
        want = [M.alu(base, bits, d, s, off) for d in ds]
        assert [int(g) for g in got] == want, (op, bits, imm)


@pytest.mark.parametrize("bits", [64, 32])
def test_neg(bits):
    ds = M.INTERESTING
    a = Asm().ldx(8, "r0", "r1", 0).neg("r0", bits=bits).exit()
    got = run_r0(a, ctx_pairs([(d, 0) for d in ds]))
    assert [int(g) for g in got] == [M.alu("neg", bits, d, 0) for d in ds]


@pytest.mark.parametrize("bits,frm", [(64, 8), (64, 16), (64, 32), (32, 8), (32, 16)])
def test_movsx(bits, frm):
    ds = M.INTERESTING
    a = Asm().ldx(8, "r2", "r1", 0).movsx("r0", "r2", frm, bits=bits).exit()
    got = run_r0(a, ctx_pairs([(d, 0) for d in ds]))
    want = [M.signed(d, frm) & M.mask(bits) for d in ds]
    assert [int(g) for g in got] == want


@pytest.mark.parametrize("order", ["le", "be", "swap"])
@pytest.mark.parametrize("width", [16, 32, 64])
def test_end(order, width):
    ds = M.INTERESTING
    a = Asm().ldx(8, "r0", "r1", 0).end("r0", width, order).exit()
    got = run_r0(a, ctx_pairs([(d, 0) for d in ds]))
    assert [int(g) for g in got] == [M.end(order, width, d) for d in ds]


JOPS = ["jeq", "jne", "jgt", "jge", "jlt", "jle", "jsgt", "jsge", "jslt", "jsle", "jset"]


@pytest.mark.parametrize("bits", [64, 32])
@pytest.mark.parametrize("op", JOPS)
def test_jump_reg(op, bits):
    a = Asm().ldx(8, "r2", "r1", 0).ldx(8, "r3", "r1", 8).mov("r0", 1)
    a.jcond(op, "r2", "r3", "end", bits=bits).mov("r0", 0).label("end").exit()
    got = run_r0(a, ctx_pairs(PAIRS))
    want = [int(M.jump(op, bits, d, s)) for d, s in PAIRS]
    assert [int(g) for g in got] == want


@pytest.mark.parametrize("bits", [64, 32])
@pytest.mark.parametrize("op", JOPS)
def test_jump_imm(op, bits):
    ds = M.INTERESTING
    ctx = ctx_pairs([(d, 0) for d in ds])
    for imm in M.INTERESTING_IMM:
        a = Asm().ldx(8, "r2", "r1", 0).mov("r0", 1)
        a.jcond(op, "r2", imm, "end", bits=bits).mov("r0", 0).label("end").exit()
        got = run_r0(a, ctx)
        want = [int(M.jump(op, bits, d, imm & M.mask(64))) for d in ds]
        assert [int(g) for g in got] == want, (op, bits, imm)


def test_ja_forms_and_ld_imm64():
    # JA with a 16-bit offset (JMP class) and with a 32-bit imm offset (JMP32 class)
    a = Asm().mov("r0", 1).ja("x").mov("r0", 2).label("x").ja("y", long=True).mov("r0", 3).label("y")
    a.ld_imm64("r2", 0xFEDCBA9876543210).add("r0", "r2").exit()
    got = run_r0(a, ctx_pairs([(0, 0)]))
    assert int(got[0]) == (1 + 0xFEDCBA9876543210) & M.mask(64)


@pytest.mark.parametrize("size", [1, 2, 4, 8])
def test_loads_zero_and_sign_extend(size):
    vals = [0, 1, 0x7F, 0x80, 0xFF, 0x7FFF, 0x8000, 0x80000000, 0xFFFFFFFF, 0x8123456789ABCDEF]
    ctx = ctx_pairs([(v, 0) for v in vals])
    a = Asm().ldx(size, "r0", "r1", 0).exit()
    assert [int(g) for g in run_r0(a, ctx)] == [v & M.mask(8 * size) for v in vals]
    if size < 8:
        a = Asm().ldx(size, "r0", "r1", 0, signed=True).exit()
        assert [int(g) for g in run_r0(a, ctx)] == [M.signed(v, 8 * size) & M.mask(64) for v in vals]


@pytest.mark.parametrize("size", [1, 2, 4, 8])
def test_store_forms_little_endian(size):
    # STX of a register and ST of a (sign-extended, truncated) immediate into a zeroed slot
    a = Asm().st(8, "r10", -8, 0).ldx(8, "r2", "r1", 0).stx(size, "r10", -8, "r2").ldx(8, "r0", "r10", -8).exit()
    v = 0x1122334455667788
    assert int(run_r0(a, ctx_pairs([(v, 0)]))[0]) == v & M.mask(8 * size)
    a = Asm().st(8, "r10", -8, 0).st(size, "r10", -8, -2).ldx(8, "r0", "r10", -8).exit()
    assert int(run_r0(a, ctx_pairs([(0, 0)]))[0]) == ((1 << 64) - 2) & M.mask(8 * size)


@pytest.mark.parametrize("size", [4, 8])
@pytest.mark.parametrize("op", ["add", "or", "and", "xor"])
@pytest.mark.parametrize("fetch", [False, True])
def test_atomics_on_stack(op, size, fetch):
    # *(stack) = a ; atomic op with b ; r0 = memory (or the fetched old value)
    pairs = PAIRS[::7]
    a = Asm().ldx(8, "r2", "r1", 0).stx(8, "r10", -8, "r2").ldx(8, "r3", "r1", 8)
    a.atomic(size, op, "r10", -8, "r3", fetch=fetch)
    if fetch:
        a.mov("r0", "r3")
    else:
        a.ldx(8, "r0", "r10", -8)
    a.exit()
    got = run_r0(a, ctx_pairs(pairs))
    m = M.mask(8 * size)
    for (d, s), g in zip(pairs, got):
        lo = {"add": (d + s) & m, "or": (d | s) & m, "and": d & s & m, "xor": (d ^ s) & m}[op]
        if fetch:
            want = d & m
        else:
            want = (d & ~m & M.mask(64)) | lo  # only the low `size` bytes change
        assert int(g) == want, (op, size, hex(d), hex(s))


@pytest.mark.parametrize("size", [4, 8])
def test_xchg_and_cmpxchg(size):
    m = M.mask(8 * size)
    pairs = PAIRS[::5]
    a = Asm().ldx(8, "r2", "r1", 0).stx(8, "r10", -8, "r2").ldx(8, "r3", "r1", 8)
    a.atomic(size, "xchg", "r10", -8, "r3").ldx(8, "r4", "r10", -8).mov("r0", "r3").xor("r0", "r4").exit()
    got = run_r0(a, ctx_pairs(pairs))
    for (d, s), g in zip(pairs, got):
        mem = (d & ~m & M.mask(64)) | (s & m)
        assert int(g) == (d & m) ^ mem
    # cmpxchg: compares r0 (low size bytes) with memory; old value goes to r0
    for expect_hit in (True, False):
        a = Asm().ldx(8, "r2", "r1", 0).stx(8, "r10", -8, "r2").ldx(8, "r3", "r1", 8)
        a.mov("r0", "r2")
        if not expect_hit:
            a.add("r0", 1)
        a.atomic(size, "cmpxchg", "r10", -8, "r3").ldx(8, "r4", "r10", -8).xor("r0", "r4").exit()
        got = run_r0(a, ctx_pairs(pairs))
        for (d, s), g in zip(pairs, got):
            mem = ((d & ~m & M.mask(64)) | (s & m)) if expect_hit else d
            assert int(g) == (d & m) ^ mem
