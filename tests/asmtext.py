"""Parser for the one-instruction-per-line assembly used by the golden fixtures.

Syntax (operands separated by spaces):
  mov r0 5 | add r0 r2 | add32 r0 1 | neg r0 | neg32 r0 | sdiv r0 3 | smod32 r0 r2
  movsx r0 r2 8 | movsx32 r0 r2 16 | end le|be|swap 16|32|64 r0
  ldx4 r0 r1 24 | ldxs2 r0 r1 0 | stx8 r10 -8 r2 | st4 r10 -4 7
  atomic8 add r0 0 r1 | atomic8 add_fetch r0 0 r1 | atomic4 xchg r10 -8 r2 | atomic8 cmpxchg r0 0 r3
  jeq r0 0 label | jgt32 r1 r2 label | ja label | jal label (32-bit offset form)
  ld_imm64 r2 0x1234 | ld_map r1 0 | call map_lookup_elem | exit | label:
"""
from __future__ import annotations

from workloads.asm import Asm


def _val(tok: str):
    if tok.startswith("r") and tok[1:].isdigit():
        return tok
    return int(tok, 0)


def assemble(lines) -> Asm:
    a = Asm()
    for raw in lines:
        line = raw.split(";")[0].strip()
        if not line:
            continue
        if line.endswith(":"):
            a.label(line[:-1])
            continue
        t = line.split()
        op, args = t[0], t[1:]
        if op == "exit":
            a.exit()
        elif op == "call":
            a.call(args[0] if not args[0][0].isdigit() else int(args[0], 0))
        elif op == "ja":
            a.ja(args[0])
        elif op == "jal":
            a.ja(args[0], long=True)
        elif op == "ld_imm64":
            a.ld_imm64(args[0], int(args[1], 0))
        elif op == "ld_map":
            a.ld_map(args[0], int(args[1], 0))
        elif op in ("neg", "neg32"):
            a.neg(args[0], bits=32 if op.endswith("32") else 64)
        elif op in ("movsx", "movsx32"):
            a.movsx(args[0], args[1], int(args[2]), bits=32 if op.endswith("32") else 64)
        elif op == "end":
            a.end(args[2], int(args[1]), args[0])
        elif op.startswith("ldxs"):
            a.ldx(int(op[4:]), args[0], args[1], int(args[2], 0), signed=True)
        elif op.startswith("ldx"):
            a.ldx(int(op[3:]), args[0], args[1], int(args[2], 0))
        elif op.startswith("stx"):
            a.stx(int(op[3:]), args[0], int(args[1], 0), args[2])
        elif op.startswith("st") and op[2:].isdigit():
            a.st(int(op[2:]), args[0], int(args[1], 0), int(args[2], 0))
        elif op.startswith("atomic"):
            size = int(op[6:])
            kind = args[0]
            fetch = kind.endswith("_fetch")
            a.atomic(size, kind.replace("_fetch", ""), args[1], int(args[2], 0), args[3], fetch=fetch)
        elif op.startswith("j"):
            bits = 32 if op.endswith("32") else 64
            name = op[:-2] if bits == 32 else op
            a.jcond(name, args[0], _val(args[1]), args[2], bits=bits)
        else:
            bits = 32 if op.endswith("32") else 64
            name = op[:-2] if bits == 32 else op
            off = 0
            if name in ("sdiv", "smod"):
                name, off = name[1:], 1
            a.alu(name, args[0], _val(args[1]), bits=bits, off=off)
    return a
