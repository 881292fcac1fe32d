"""Independent Python big-integer model of eBPF arithmetic and comparisons.

Written from the standard eBPF ISA (RFC 9669 Sec. 4.1 arithmetic, Sec. 4.2 byte swaps,
Sec. 4.3 jump conditions) with Python's unbounded integers, so that it shares no code
and no idiom with the C oracle it pins.  Signed division truncates toward zero
(RFC 9669 Sec. 4.1); the overflow case INT_MIN / -1 wraps to INT_MIN and INT_MIN % -1
is 0, which is what exact arithmetic reduced modulo 2^n gives.
"""
from __future__ import annotations


def mask(bits: int) -> int:
    return (1 << bits) - 1


def signed(v: int, bits: int) -> int:
    v &= mask(bits)
    return v - (1 << bits) if v >= (1 << (bits - 1)) else v


def trunc_div(a: int, b: int) -> int:
    q = abs(a) // abs(b)
    return q if (a >= 0) == (b >= 0) else -q


def alu(op: str, bits: int, d: int, s: int, off: int = 0) -> int:
    """Result (as an unsigned 64-bit integer) of `dst op= src` for ALU64 (bits=64) or ALU (bits=32)."""
    m = mask(bits)
    a, b = d & m, s & m
    if op == "add":
        r = a + b
    elif op == "sub":
        r = a - b
    elif op == "mul":
        r = a * b
    elif op == "div":
        if off == 0:
            r = a // b if b else 0
        else:
            sa, sb = signed(a, bits), signed(b, bits)
            r = trunc_div(sa, sb) if sb else 0
    elif op == "mod":
        if off == 0:
            r = a % b if b else a
        else:
            sa, sb = signed(a, bits), signed(b, bits)
            r = sa - sb * trunc_div(sa, sb) if sb else sa
    elif op == "or":
        r = a | b
    elif op == "and":
        r = a & b
    elif op == "xor":
        r = a ^ b
    elif op == "lsh":
        r = a << (b % bits)
    elif op == "rsh":
        r = a >> (b % bits)
    elif op == "arsh":
        r = signed(a, bits) >> (b % bits)
    elif op == "neg":
        r = -a
    elif op == "mov":
        r = b if off == 0 else signed(s, off)
    else:
        raise ValueError(op)
    return r & m  # ALU (32-bit) results are zero-extended into the 64-bit register


def byteswap(v: int, width: int) -> int:
    bs = (v & mask(width)).to_bytes(width // 8, "little")
    return int.from_bytes(bs, "big")


def end(order: str, width: int, d: int) -> int:
    """to-le on a little-endian machine truncates; to-be and swap reverse the low bytes."""
    if order == "le":
        return d & mask(width)
    return byteswap(d, width)


def jump(op: str, bits: int, d: int, s: int) -> bool:
    a, b = d & mask(bits), s & mask(bits)
    sa, sb = signed(a, bits), signed(b, bits)
    return {
        "jeq": a == b, "jne": a != b, "jgt": a > b, "jge": a >= b, "jlt": a < b, "jle": a <= b,
        "jsgt": sa > sb, "jsge": sa >= sb, "jslt": sa < sb, "jsle": sa <= sb, "jset": (a & b) != 0,
    }[op]


INTERESTING = [
    0, 1, 2, 3, 7, 8, 31, 32, 33, 63, 64, 65, 0x7F, 0x80, 0xFF, 0x7FFF, 0x8000, 0xFFFF,
    0x7FFFFFFF, 0x80000000, 0xFFFFFFFF, 1 << 32, (1 << 32) + 5, 0x123456789ABCDEF0,
    (1 << 63) - 1, 1 << 63, (1 << 64) - 1, (1 << 64) - 2, (1 << 64) - 7, (1 << 64) - 0x80000000,
]
INTERESTING_IMM = [0, 1, 2, 7, 31, 32, 63, 64, 65, 0x7F, 0x80, 0x7FFF, -1, -2, -7, -0x80000000, 0x7FFFFFFF, 12345]
