"""LocPIR circuits over gates -- TEST INFRASTRUCTURE ONLY (part of the oracle).

A circuit is built as a netlist of gates over numbered wires, then evaluated either
on plaintext bits (to check the circuit logic against integer truth) or on
ciphertexts through the C oracle's gates.  Gates are pure functions of their input
ciphertexts, so evaluating independent gates together (one oracle batch per
bootstrap level and gate kind) gives the same ciphertexts as any other
topological order.

Followed passages (LocPIR, arXiv 2407.19871):
  * HomCompS: Algorithm 2 (Section 4.2) -- t0 = Enc(0); flip both MSBs; for each bit
    from index 0 (least significant) up: t1 = XNOR(c1[i], c2[i]); t0 = MUX(t1, t0, c2[i]).
  * HomCompLE: the negation of HomCompS (Section 4.2), read as NOT(HomCompS(b, a)), i.e. a <= b.
  * LocPIR: Algorithm 3 (Section 4.3) -- four comparisons per box, three HomANDs,
    bitwiseAND (Algorithm 5) of the validation bit with the box's service, then the sum.
  * HomAddXOR: Algorithm 4 (Section 4.4); its body's assignment to S_i[j] is read as
    S[j].  The default combine is a pairwise XOR tree over boxes.
Beyond the paper: comp_s_known / locpir_known, the same circuits when the server knows
the box bounds in the clear (a comparator then costs at most l - 1 bootstraps, not 3l).
Readings where the paper is silent or garbled are listed in the design notes.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import AND, MUX, NOT, OR, XNOR, XOR, NAND, Keys, gate_batch, trivial

CONST = -1   # pseudo-op: trivial constant, ins = (bit,)
INPUT = -2   # pseudo-op: circuit input


@dataclass
class Netlist:
    ops: list[int] = field(default_factory=list)
    ins: list[tuple] = field(default_factory=list)

    def _new(self, op: int, ins: tuple) -> int:
        self.ops.append(op)
        self.ins.append(ins)
        return len(self.ops) - 1

    def input(self) -> int:
        return self._new(INPUT, ())

    def inputs(self, k: int) -> list[int]:
        return [self.input() for _ in range(k)]

    def const(self, bit: int) -> int:
        return self._new(CONST, (int(bit),))

    def gate(self, op: int, *ins: int) -> int:
        return self._new(op, tuple(ins))

    def NOT(self, w: int) -> int:
        return self.gate(NOT, w)

    def bootstraps(self) -> tuple[int, int]:
        """(blind rotations, key switches) the netlist costs."""
        br = sum(2 if o == MUX else 1 for o in self.ops if o >= 0 and o != NOT)
        ks = sum(1 for o in self.ops if o >= 0 and o != NOT)
        return br, ks


# ---------------------------------------------------------------------------
# Circuit builders.
# ---------------------------------------------------------------------------

def comp_s(net: Netlist, c1: list[int], c2: list[int], signed: bool) -> int:
    """HomCompS (Algorithm 2): encrypts 1 iff x1 < x2; bits least significant first."""
    l = len(c1)
    c1, c2 = list(c1), list(c2)
    t0 = net.const(0)
    if signed:
        c1[l - 1] = net.NOT(c1[l - 1])
        c2[l - 1] = net.NOT(c2[l - 1])
    for i in range(l):
        t1 = net.gate(XNOR, c1[i], c2[i])
        t0 = net.gate(MUX, t1, t0, c2[i])
    return t0


def comp_le(net: Netlist, a: list[int], b: list[int], signed: bool) -> int:
    """HomCompLE: a <= b, as the negation of HomCompS(b, a)."""
    return net.NOT(comp_s(net, b, a, signed))


def comp_s_known(net: Netlist, c1: list[int], K: int, signed: bool) -> int:
    """HomCompS with a server-known second operand (beyond the paper): encrypts 1 iff
    x1 < K.  Algorithm 2's steps with c2 replaced by the plaintext bits k_i of K:
    XNOR(a, k) is a for k = 1 and NOT a for k = 0, and MUX(t1, t0, k) = t1 ? t0 : k is
    AND(NOT a, t0) for k = 0 and OR(NOT a, t0) for k = 1.  While t0 is still a known
    constant c, the step keeps c when k = c and yields NOT a otherwise, with no gate.
    A constant result is returned as a trivial constant wire."""
    l = len(c1)
    cst, t0 = 0, None
    for i in range(l):
        a = c1[i]
        k = (K >> i) & 1
        if signed and i == l - 1:
            a = net.NOT(a)
            k ^= 1
        na = net.NOT(a)
        if t0 is None:
            if k != cst:
                t0 = na
        else:
            t0 = net.gate(OR if k else AND, na, t0)
    return net.const(cst) if t0 is None else t0


XOR_TREE, XOR_CHAIN, OR_TREE = 0, 1, 2


def _tree(net: Netlist, op: int, rows: list[list[int]]) -> list[int]:
    while len(rows) > 1:
        nxt = []
        for i in range(0, len(rows) - 1, 2):
            nxt.append([net.gate(op, u, v) for u, v in zip(rows[i], rows[i + 1])])
        if len(rows) % 2:
            nxt.append(rows[-1])
        rows = nxt
    return rows[0]


def locpir(net: Netlist, x: list[int], y: list[int], boxes: list[tuple[list[int], ...]],
           services: list[list[int]], comb: int = XOR_TREE, signed: bool = False) -> list[int]:
    """LocPIR (Algorithm 3) over B_x boxes; box = (X1, X2, Y1, Y2) bit wires, the point
    is inside iff X1 <= x < X2 and Y1 <= y < Y2."""
    per_box = []
    for (X1, X2, Y1, Y2), svc in zip(boxes, services):
        xl = comp_le(net, X1, x, signed)
        xr = comp_s(net, x, X2, signed)
        yl = comp_le(net, Y1, y, signed)
        yr = comp_s(net, y, Y2, signed)
        v1 = net.gate(AND, xl, xr)
        v2 = net.gate(AND, yl, yr)
        f = net.gate(AND, v1, v2)
        per_box.append([net.gate(AND, f, s) for s in svc])  # bitwiseAND, Algorithm 5
    if comb == XOR_CHAIN:
        m = len(services[0])
        S = [net.const(0) for _ in range(m)]
        for Si in per_box:
            S = [net.gate(XOR, S[j], Si[j]) for j in range(m)]
        return S
    return _tree(net, OR if comb == OR_TREE else XOR, per_box)


def locpir_known(net: Netlist, x: list[int], y: list[int], bounds: list[tuple[int, int, int, int]],
                 services: list[list[int]], comb: int = XOR_TREE, signed: bool = False) -> list[int]:
    """LocPIR with server-known box bounds (X1, X2, Y1, Y2) (beyond the paper): the four
    comparisons of Algorithm 3 become X1 <= x = NOT(x < X1), x < X2, and the same for y,
    each by comp_s_known; validation, bitwiseAND and the combine are Algorithm 3's."""
    per_box = []
    for (X1, X2, Y1, Y2), svc in zip(bounds, services):
        xl = net.NOT(comp_s_known(net, x, X1, signed))
        xr = comp_s_known(net, x, X2, signed)
        yl = net.NOT(comp_s_known(net, y, Y1, signed))
        yr = comp_s_known(net, y, Y2, signed)
        v1 = net.gate(AND, xl, xr)
        v2 = net.gate(AND, yl, yr)
        f = net.gate(AND, v1, v2)
        per_box.append([net.gate(AND, f, s) for s in svc])
    if comb == XOR_CHAIN:
        m = len(services[0])
        S = [net.const(0) for _ in range(m)]
        for Si in per_box:
            S = [net.gate(XOR, S[j], Si[j]) for j in range(m)]
        return S
    return _tree(net, OR if comb == OR_TREE else XOR, per_box)


# ---------------------------------------------------------------------------
# Evaluation.
# ---------------------------------------------------------------------------

_PLAIN = {
    NAND: lambda a, b: 1 - (a & b),
    AND: lambda a, b: a & b,
    OR: lambda a, b: a | b,
    XOR: lambda a, b: a ^ b,
    XNOR: lambda a, b: 1 - (a ^ b),
}


def eval_plain(net: Netlist, inputs: dict[int, int]) -> list[int]:
    """Evaluate on plaintext bits; inputs maps input wire -> bit."""
    val = [0] * len(net.ops)
    for w, (op, ins) in enumerate(zip(net.ops, net.ins)):
        if op == INPUT:
            val[w] = int(inputs[w])
        elif op == CONST:
            val[w] = ins[0]
        elif op == NOT:
            val[w] = 1 - val[ins[0]]
        elif op == MUX:
            val[w] = val[ins[1]] if val[ins[0]] else val[ins[2]]
        else:
            val[w] = _PLAIN[op](val[ins[0]], val[ins[1]])
    return val


def depths(net: Netlist) -> list[int]:
    """Bootstrap depth of each wire (NOT, constants and inputs cost nothing)."""
    d = [0] * len(net.ops)
    for w, (op, ins) in enumerate(zip(net.ops, net.ins)):
        if op in (INPUT, CONST):
            d[w] = 0
        elif op == NOT:
            d[w] = d[ins[0]]
        else:
            d[w] = 1 + max(d[i] for i in ins)
    return d


def eval_encrypted(net: Netlist, keys: Keys, inputs: dict[int, np.ndarray],
                   nthreads: int | None = None) -> np.ndarray:
    """Evaluate on ciphertexts; returns [wires][n+1] (unevaluated wires stay 0)."""
    n = keys.params.n
    val = np.zeros((len(net.ops), n + 1), np.uint32)
    d = depths(net)
    for w, op in enumerate(net.ops):
        if op == INPUT:
            val[w] = inputs[w]
        elif op == CONST:
            val[w] = trivial(net.ins[w][0], n)
    for level in range(0, max(d) + 1 if d else 1):
        if level > 0:
            for op in (NAND, AND, OR, XOR, XNOR, MUX):
                ws = [w for w in range(len(net.ops)) if net.ops[w] == op and d[w] == level]
                if not ws:
                    continue
                a = val[[net.ins[w][0] for w in ws]]
                b = val[[net.ins[w][1] for w in ws]]
                c = val[[net.ins[w][2] for w in ws]] if op == MUX else None
                val[ws] = gate_batch(keys, op, a, b, c, nthreads)
        for w in range(len(net.ops)):
            if net.ops[w] == NOT and d[w] == level:
                val[w] = ((-val[net.ins[w][0]].astype(np.int64)) & 0xFFFFFFFF).astype(np.uint32)
    return val
