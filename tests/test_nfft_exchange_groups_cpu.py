"""The register NFFT kernel's pass structure (Sec. 3 recursion, radix-2 stages
grouped three at a time) and the scope of its barriers, checked by brute
force on the CPU.

A thread of a 2^L-point (sub-)vector holds 8 points.  In a pass with index
window W its positions are base | j << W, j < 8, with base = (t mod 2^W) |
(t >> W) << (W + 3); the pass that touches global memory in bit-reversed
order (the first DIT pass, the last DIF pass) takes positions 8 rev(t) + j
instead.  DIT windows ascend (0, 3, ..., the last clamped to L - 3); DIF
windows descend (the first at L - 3 taking the top L mod 3 stages when that
is not 0, then 3-stage windows down to 0).

Claims: every pass covers each position exactly once, every stage lies in
exactly one pass's window, and a position's writer and reader in
consecutive passes share their thread index above bit log2 G with G = 2^W of
the reader's window (DIT, writer not bit-reversed) or of the writer's (DIF,
reader not bit-reversed) -- so the exchange between those passes needs a
barrier over groups of G threads only.
"""
import pytest


def _bitrev(x, n):
    return int(format(x, f"0{n}b")[::-1], 2) if n else 0


def _dit_passes(L):
    out, b0 = [], 0
    while b0 < L:
        W = b0 if b0 + 3 <= L else L - 3
        out.append({"W": W, "stages": range(b0, min(b0 + 3, L)), "rev": b0 == 0})
        b0 += 3
    return out


def _dif_passes(L):
    out, b1 = [], L
    while b1 > 0:
        first = b1 == L
        W = b1 - 3 if b1 >= 3 else 0
        lo = L - L % 3 if (first and L % 3) else W
        out.append({"W": W, "stages": range(lo, b1), "rev": lo == 0})
        b1 = lo
    return out


def _positions(L, p, t):
    if p["rev"]:
        return [8 * _bitrev(t, L - 3) + j for j in range(8)]
    W = p["W"]
    base = (t & ((1 << W) - 1)) | ((t >> W) << (W + 3))
    return [base | (j << W) for j in range(8)]


def _owner(L, p):
    own = {}
    for t in range(1 << (L - 3)):
        for q in _positions(L, p, t):
            assert q not in own
            own[q] = t
    assert sorted(own) == list(range(1 << L))
    return own


@pytest.mark.parametrize("L", range(3, 13))
@pytest.mark.parametrize("dif", [False, True])
def test_passes_cover_positions_and_stages(L, dif):
    passes = _dif_passes(L) if dif else _dit_passes(L)
    stages = [b for p in passes for b in p["stages"]]
    assert sorted(stages) == list(range(L))
    for p in passes:
        _owner(L, p)
        # each stage of the pass pairs two of the thread's own points
        assert all(p["W"] <= b < p["W"] + 3 for b in p["stages"])


@pytest.mark.parametrize("L", range(3, 13))
@pytest.mark.parametrize("dif", [False, True])
def test_exchange_closes_over_thread_groups(L, dif):
    passes = _dif_passes(L) if dif else _dit_passes(L)
    tpv = 1 << (L - 3)
    local = 0
    for w, r in zip(passes, passes[1:]):
        if dif:
            G = tpv if r["rev"] else 1 << w["W"]
        else:
            G = tpv if w["rev"] else 1 << r["W"]
        if G >= tpv:
            continue
        ow, orr = _owner(L, w), _owner(L, r)
        assert all(ow[q] // G == orr[q] // G for q in range(1 << L))
        local += 1
    # the transitions that close over groups smaller than the (sub-)vector
    assert local == (1 if L in (10, 11, 12) else 0)
