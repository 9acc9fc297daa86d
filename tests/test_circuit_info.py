"""The library's host-side circuit builder and level scheduler against the oracle's netlists
(CPU, no GPU): lp_circuit_info reports, for one LocPIR query, the bootstrapped gates per
kind, blind rotations, key switches, the number of bootstrap levels and the widest level,
as the library builds the circuit for its batch entry points, plans and server.  Each figure
must equal the same count taken from the oracle's independently built netlist (Algorithms
2-5, and the server-known-bounds variant), and the closed forms of the gate-count formula."""
import math

import numpy as np
import pytest

import synth
from oracle import MUX, NOT
from oracle import circuits as C


def _lib_info(*args, **kw):
    from paper_2407_19871_gb300 import locpir
    return locpir.lp_circuit_info(*args, **kw)


def _oracle_info(l, signed, nb, m, comb, bounds=None):
    net = C.Netlist()
    x, y = net.inputs(l), net.inputs(l)
    sw = [net.inputs(m) for _ in range(nb)]
    if bounds is None:
        bw = [tuple(net.inputs(l) for _ in range(4)) for _ in range(nb)]
        C.locpir(net, x, y, bw, sw, comb, signed)
    else:
        C.locpir_known(net, x, y, [tuple(int(v) for v in b) for b in bounds], sw, comb, signed)
    by_op = [0] * 8
    for op in net.ops:
        if op >= 0 and op != NOT:
            by_op[op] += 1
    br, ks = net.bootstraps()
    d = C.depths(net)
    per_level = {}
    for w, op in enumerate(net.ops):
        if op >= 0 and op != NOT:
            per_level[d[w]] = per_level.get(d[w], 0) + (2 if op == MUX else 1)
    return {"gates_by_op": by_op, "blind_rotations": br, "key_switches": ks,
            "levels": len(per_level), "widest_level": max(per_level.values(), default=0),
            "depth": max(d)}


def _same(got, want, what):
    for k in ("gates_by_op", "blind_rotations", "key_switches", "levels", "widest_level"):
        assert got[k] == want[k], f"{what}: {k} library {got[k]} oracle {want[k]}"


@pytest.mark.parametrize("comb", [C.XOR_TREE, C.XOR_CHAIN, C.OR_TREE])
@pytest.mark.parametrize("signed", [False, True])
def test_encrypted_bounds_match_oracle_netlist(comb, signed):
    for l, nb, m in [(1, 1, 1), (2, 3, 2), (4, 1, 4), (13, 9, 9), (16, 10, 9), (16, 28, 128), (32, 1, 256),
                     (24, 5, 8), (64, 2, 3)]:
        _same(_lib_info(l, signed, nb, m, comb), _oracle_info(l, signed, nb, m, comb),
              f"l={l} B_x={nb} m={m} comb={comb} signed={signed}")


@pytest.mark.parametrize("comb", [C.XOR_TREE, C.XOR_CHAIN, C.OR_TREE])
@pytest.mark.parametrize("signed", [False, True])
def test_known_bounds_match_oracle_netlist(comb, signed):
    """Server-known bounds: random bounds (seeded), plus the edge values 0, 1, 2^(l-1) and
    2^l - 1 whose comparators need no gate or a single one."""
    for l, nb, m in [(1, 2, 1), (4, 3, 4), (8, 5, 3), (16, 9, 9), (32, 4, 16), (64, 2, 2)]:
        d = synth.splitmix64(11, l * 100 + nb, 4 * nb)
        mask = (1 << l) - 1
        bounds = (d & np.uint64(mask)).reshape(nb, 4)
        edges = np.array([[0, 1, (1 << (l - 1)), mask]], dtype=np.uint64)
        bounds = np.concatenate([bounds, edges])
        n = nb + 1
        _same(_lib_info(l, signed, n, m, comb, bounds=bounds), _oracle_info(l, signed, n, m, comb, bounds),
              f"known l={l} B_x={n} m={m} comb={comb} signed={signed}")


@pytest.mark.parametrize("l,nb,m", [(13, 9, 9), (16, 1, 64), (32, 1, 256), (16, 10, 9), (8, 28, 128)])
def test_closed_forms(l, nb, m):
    """XOR tree: per box 12l + 3 + m blind rotations and 8l + 3 + m key switches, plus
    (B_x - 1) m for the combine; l + 1 comparator levels, 2 validation levels, one service
    level and ceil(log2 B_x) combine levels.  The first level holds every XNOR: 4l per box,
    each one blind rotation."""
    s = _lib_info(l, False, nb, m, C.XOR_TREE)
    assert s["blind_rotations"] == nb * (12 * l + 3 + m) + (nb - 1) * m
    assert s["key_switches"] == nb * (8 * l + 3 + m) + (nb - 1) * m
    assert s["levels"] == l + 1 + 2 + 1 + math.ceil(math.log2(nb))
    assert s["gates_by_op"][C.XNOR] == 4 * l * nb and s["gates_by_op"][MUX] == 4 * l * nb
    assert s["widest_level"] == max(4 * l * nb, nb * m, 8 * nb)
    # Wires: the inputs, one per bootstrapped gate and the shared trivial zero (Enc(0) of
    # Algorithm 2) -- the closed form the query server reserves pool space with.
    assert s["wires"] == 2 * l + 4 * l * nb + m * nb + s["key_switches"] + 1
    chain = _lib_info(l, False, nb, m, C.XOR_CHAIN)
    assert chain["blind_rotations"] == nb * (12 * l + 3 + m) + nb * m
    assert chain["levels"] == l + 1 + 2 + 1 + nb


def test_known_bounds_cost_at_most_l_minus_1_per_comparator():
    for l in (4, 16, 32):
        mask = (1 << l) - 1
        bounds = np.array([[1, mask, 3, mask - 1]], dtype=np.uint64)
        s = _lib_info(l, False, 1, 1, C.XOR_TREE, bounds=bounds)
        enc = _lib_info(l, False, 1, 1, C.XOR_TREE)
        assert s["blind_rotations"] <= 4 * (l - 1) + 3 + 1 < enc["blind_rotations"]


@pytest.mark.parametrize("args", [(0, 0, 1, 1, 0), (65, 0, 1, 1, 0), (16, 0, 0, 1, 0), (16, 0, 1, 0, 0),
                                  (16, 0, 1, 1, 3)])
def test_invalid_shapes_are_rejected(args):
    from paper_2407_19871_gb300 import locpir
    with pytest.raises(locpir.LocpirError) as e:
        _lib_info(*args)
    assert e.value.code == locpir.LP_EINVAL
