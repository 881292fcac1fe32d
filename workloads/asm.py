"""Tiny eBPF assembler: turns a readable instruction list into raw 8-byte eBPF slots.

Input-side tooling shared by the oracle tests and the engine tests. It only *encodes*
instructions (opcode byte, register nibbles, 16-bit offset, 32-bit immediate) following
the standard eBPF instruction encoding (RFC 9669, Sec. 3 "Instruction encoding"); it
carries none of the execution semantics.

The paper's policies are authored with clang/libbpf (Sec. 4.2, "User-space Control
Plane"); here programs are assembled directly so that tests can state every
instruction they run.
"""
from __future__ import annotations

import struct
from typing import Dict, List, Optional, Tuple, Union

import numpy as np

# ---- instruction classes (RFC 9669 Sec. 3.3) ----
LD, LDX, ST, STX, ALU, JMP, JMP32, ALU64 = range(8)
# ---- source bit ----
K, X = 0x00, 0x08
# ---- ALU operation codes (high nibble) ----
ALU_OPS = {
    "add": 0x00, "sub": 0x10, "mul": 0x20, "div": 0x30, "or": 0x40, "and": 0x50,
    "lsh": 0x60, "rsh": 0x70, "neg": 0x80, "mod": 0x90, "xor": 0xA0, "mov": 0xB0,
    "arsh": 0xC0, "end": 0xD0,
}
# ---- jump operation codes (high nibble) ----
JMP_OPS = {
    "ja": 0x00, "jeq": 0x10, "jgt": 0x20, "jge": 0x30, "jset": 0x40, "jne": 0x50,
    "jsgt": 0x60, "jsge": 0x70, "call": 0x80, "exit": 0x90, "jlt": 0xA0, "jle": 0xB0,
    "jslt": 0xC0, "jsle": 0xD0,
}
# ---- load/store modes and sizes (RFC 9669 Sec. 5) ----
MODE_IMM, MODE_ABS, MODE_IND, MODE_MEM, MODE_MEMSX, MODE_ATOMIC = 0x00, 0x20, 0x40, 0x60, 0x80, 0xC0
SIZES = {1: 0x10, 2: 0x08, 4: 0x00, 8: 0x18}
# ---- atomic immediates (RFC 9669 Sec. 5.3) ----
ATOMIC_OPS = {"add": 0x00, "or": 0x40, "and": 0x50, "xor": 0xA0}
FETCH = 0x01
XCHG = 0xE0 | FETCH
CMPXCHG = 0xF0 | FETCH

# ---- helper ids (Linux UAPI numbering) and engine-private helpers ----
HELPER = {
    "map_lookup_elem": 1,
    "map_update_elem": 2,
    "map_delete_elem": 3,
    "ringbuf_output": 130,
    "ringbuf_reserve": 131,
    "ringbuf_submit": 132,
    "ringbuf_discard": 133,
    "atomic_max_u64": 0x10000,
    "atomic_min_u64": 0x10001,
    # warp-level aggregation (SIMT verification only): u64 (u64 v) reduced over the warp's lanes
    "warp_sum_u64": 0x10010,
    "warp_max_u64": 0x10011,
    "warp_min_u64": 0x10012,
    "warp_or_u64": 0x10013,
    "warp_and_u64": 0x10014,
    "warp_count": 0x10015,
}
BPF_ANY, BPF_NOEXIST, BPF_EXIST = 0, 1, 2
PSEUDO_MAP_FD = 1

# ---- map types (Linux enum bpf_map_type values) ----
MAP_HASH, MAP_ARRAY, MAP_RINGBUF = 1, 2, 27


def _reg(r: Union[int, str]) -> int:
    if isinstance(r, str):
        assert r[0] == "r", r
        r = int(r[1:])
    assert 0 <= r <= 15, r
    return r


def encode(opcode: int, dst: int = 0, src: int = 0, off: int = 0, imm: int = 0) -> int:
    """One 64-bit slot, little-endian field order: opcode, regs, off, imm."""
    assert 0 <= opcode <= 0xFF
    off &= 0xFFFF
    imm &= 0xFFFFFFFF
    return opcode | ((dst & 0xF) << 8) | ((src & 0xF) << 12) | (off << 16) | (imm << 32)


Operand = Union[int, str]


class Asm:
    """Label-aware builder; `prog()` returns a uint64 numpy array of slots."""

    def __init__(self) -> None:
        self.slots: List[int] = []
        self.labels: Dict[str, int] = {}
        self.fixups: List[Tuple[int, str, str]] = []  # (slot, label, kind)

    # -- bookkeeping --
    def label(self, name: str) -> "Asm":
        assert name not in self.labels, name
        self.labels[name] = len(self.slots)
        return self

    def raw(self, opcode: int, dst: int = 0, src: int = 0, off: int = 0, imm: int = 0) -> "Asm":
        self.slots.append(encode(opcode, dst, src, off, imm))
        return self

    def __len__(self) -> int:
        return len(self.slots)

    # -- ALU --
    def alu(self, op: str, dst: Operand, src: Operand, *, bits: int = 64, off: int = 0) -> "Asm":
        cls = ALU64 if bits == 64 else ALU
        if isinstance(src, str):
            return self.raw(cls | X | ALU_OPS[op], _reg(dst), _reg(src), off, 0)
        return self.raw(cls | K | ALU_OPS[op], _reg(dst), 0, off, int(src))

    def mov(self, dst: Operand, src: Operand, bits: int = 64) -> "Asm":
        return self.alu("mov", dst, src, bits=bits)

    def movsx(self, dst: Operand, src: Operand, from_bits: int, bits: int = 64) -> "Asm":
        return self.alu("mov", dst, src, bits=bits, off=from_bits)

    def sdiv(self, dst: Operand, src: Operand, bits: int = 64) -> "Asm":
        return self.alu("div", dst, src, bits=bits, off=1)

    def smod(self, dst: Operand, src: Operand, bits: int = 64) -> "Asm":
        return self.alu("mod", dst, src, bits=bits, off=1)

    def neg(self, dst: Operand, bits: int = 64) -> "Asm":
        cls = ALU64 if bits == 64 else ALU
        return self.raw(cls | K | ALU_OPS["neg"], _reg(dst))

    def end(self, dst: Operand, width: int, order: str) -> "Asm":
        """order: 'le' / 'be' (ALU class) or 'swap' (ALU64 class, unconditional)."""
        if order == "swap":
            return self.raw(ALU64 | K | ALU_OPS["end"], _reg(dst), 0, 0, width)
        return self.raw(ALU | (X if order == "be" else K) | ALU_OPS["end"], _reg(dst), 0, 0, width)

    def __getattr__(self, name: str):
        # add/sub/mul/... and their 32-bit forms add32/sub32/...
        base, bits = (name[:-2], 32) if name.endswith("32") else (name, 64)
        if base in ALU_OPS and base not in ("neg", "end"):
            return lambda dst, src: self.alu(base, dst, src, bits=bits)
        if base in JMP_OPS and base not in ("call", "exit", "ja"):
            return lambda dst, src, target: self.jcond(base, dst, src, target, bits=bits)
        raise AttributeError(name)

    # -- 64-bit immediate loads --
    def ld_imm64(self, dst: Operand, value: int) -> "Asm":
        value &= (1 << 64) - 1
        self.raw(LD | MODE_IMM | 0x18, _reg(dst), 0, 0, value & 0xFFFFFFFF)
        return self.raw(0, 0, 0, 0, value >> 32)

    def ld_map(self, dst: Operand, map_index: int) -> "Asm":
        self.raw(LD | MODE_IMM | 0x18, _reg(dst), PSEUDO_MAP_FD, 0, map_index)
        return self.raw(0, 0, 0, 0, 0)

    # -- memory --
    def ldx(self, size: int, dst: Operand, src: Operand, off: int, signed: bool = False) -> "Asm":
        mode = MODE_MEMSX if signed else MODE_MEM
        return self.raw(LDX | mode | SIZES[size], _reg(dst), _reg(src), off, 0)

    def stx(self, size: int, dst: Operand, off: int, src: Operand) -> "Asm":
        return self.raw(STX | MODE_MEM | SIZES[size], _reg(dst), _reg(src), off, 0)

    def st(self, size: int, dst: Operand, off: int, imm: int) -> "Asm":
        return self.raw(ST | MODE_MEM | SIZES[size], _reg(dst), 0, off, imm)

    def atomic(self, size: int, op: str, dst: Operand, off: int, src: Operand, fetch: bool = False) -> "Asm":
        if op == "xchg":
            imm = XCHG
        elif op == "cmpxchg":
            imm = CMPXCHG
        else:
            imm = ATOMIC_OPS[op] | (FETCH if fetch else 0)
        return self.raw(STX | MODE_ATOMIC | SIZES[size], _reg(dst), _reg(src), off, imm)

    # -- control flow --
    def jcond(self, op: str, dst: Operand, src: Operand, target: str, bits: int = 64) -> "Asm":
        cls = JMP if bits == 64 else JMP32
        slot = len(self.slots)
        if isinstance(src, str):
            self.raw(cls | X | JMP_OPS[op], _reg(dst), _reg(src), 0, 0)
        else:
            self.raw(cls | K | JMP_OPS[op], _reg(dst), 0, 0, int(src))
        self.fixups.append((slot, target, "off"))
        return self

    def ja(self, target: str, long: bool = False) -> "Asm":
        slot = len(self.slots)
        if long:  # JMP32-class JA: the offset lives in imm
            self.raw(JMP32 | JMP_OPS["ja"])
            self.fixups.append((slot, target, "imm"))
        else:
            self.raw(JMP | JMP_OPS["ja"])
            self.fixups.append((slot, target, "off"))
        return self

    def call(self, helper: Union[int, str]) -> "Asm":
        hid = HELPER[helper] if isinstance(helper, str) else int(helper)
        return self.raw(JMP | JMP_OPS["call"], 0, 0, 0, hid)

    def exit(self) -> "Asm":
        return self.raw(JMP | JMP_OPS["exit"])

    # -- output --
    def prog(self) -> np.ndarray:
        slots = list(self.slots)
        for slot, target, kind in self.fixups:
            assert target in self.labels, f"undefined label {target}"
            rel = self.labels[target] - (slot + 1)
            op = slots[slot] & 0xFF
            dst = (slots[slot] >> 8) & 0xF
            src = (slots[slot] >> 12) & 0xF
            off = (slots[slot] >> 16) & 0xFFFF
            imm = slots[slot] >> 32
            if kind == "off":
                assert -32768 <= rel <= 32767
                off = rel
            else:
                imm = rel
            slots[slot] = encode(op, dst, src, off, imm)
        return np.array(slots, dtype=np.uint64)


def decode_fields(slot: int) -> Tuple[int, int, int, int, int]:
    """(opcode, dst, src, off signed, imm signed) of one raw slot."""
    slot = int(slot)
    op = slot & 0xFF
    dst = (slot >> 8) & 0xF
    src = (slot >> 12) & 0xF
    off = struct.unpack("<h", struct.pack("<H", (slot >> 16) & 0xFFFF))[0]
    imm = struct.unpack("<i", struct.pack("<I", (slot >> 32) & 0xFFFFFFFF))[0]
    return op, dst, src, off, imm


def from_bytes(blob: bytes) -> np.ndarray:
    assert len(blob) % 8 == 0
    return np.frombuffer(blob, dtype="<u8").astype(np.uint64)


def prog_or_none(p: Optional[Asm]) -> Optional[np.ndarray]:
    return None if p is None else p.prog()
