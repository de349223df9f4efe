"""The batch schedule and tile-width policies on the host (no GPU)."""
import pytest

import workloads as W
from paper_1611_00860_gb300 import _lib as H


def _grid(M, N, bn, tm=128):
    return {(m0, n0) for m0 in range(0, M, tm) for n0 in range(0, N, bn)}


@pytest.mark.parametrize("policy", range(12))
def test_schedule_covers_every_tile_once(policy):
    # policies 4-11: 256-row tiles on CTA pairs, the units half as many
    shapes = W.batched_shapes(64, seed=5)
    M, N, K = zip(*shapes)
    bn, slots = H.hpvm_batch_plan(M, N, K, policy)
    tm = 256 if policy >= 4 else 128
    tiles = [t for t in slots if t[0] >= 0]
    assert len(tiles) == len(set(tiles))
    for i, (m, n, _k) in enumerate(shapes):
        got = {(t[1], t[2]) for t in tiles if t[0] == i}
        assert got == _grid(m, n, bn[i], tm)
    # CTA u runs slots u, u + G, ...; each CTA's tiles longest first, and
    # the CTAs' loads (longest-first to the least loaded) differ by at most
    # one tile's cost
    G = max(t[3] for t in slots) + 1
    assert len(slots) % G == 0 and all(t[3] == p % G for p, t in enumerate(slots))
    cost = lambda t: ((K[t[0]] + 127) // 128 * 128) * bn[t[0]] * (tm // 128) + 4096
    loads = []
    for u in range(G):
        c = [cost(t) for t in slots[u::G] if t[0] >= 0]
        assert all(a >= b for a, b in zip(c, c[1:]))
        loads.append(sum(c))
    assert max(loads) - min(loads) <= max(cost(t) for t in tiles)


def test_policies():
    M, N, K = [300, 300, 2048], [40, 1000, 100], [512, 512, 64]
    assert H.hpvm_batch_plan(M, N, K, 0)[0] == [256, 256, 256]
    assert H.hpvm_batch_plan(M, N, K, 1)[0] == [128, 128, 128]
    bn2 = H.hpvm_batch_plan(M, N, K, 2)[0]
    assert bn2[0] == 64   # 40 columns: the narrowest tile wastes the least
    assert bn2[1] == 256  # 1000 columns: wide tiles
    # a heavier per-tile overhead never asks for more tiles than a lighter one
    bn3 = H.hpvm_batch_plan(M, N, K, 3)[0]
    assert all(b3 >= b2 for b2, b3 in zip(bn2, bn3))
    # the pair policies apply the same rules to 256-row tiles
    assert H.hpvm_batch_plan(M, N, K, 4)[0] == [256, 256, 256]
    assert H.hpvm_batch_plan(M, N, K, 5)[0] == [128, 128, 128]
    assert H.hpvm_batch_plan(M, N, K, 6)[0][0] == 64


def test_pair_policies_halve_the_units():
    shapes = W.batched_shapes(64, seed=5)
    M, N, K = zip(*shapes)
    g1 = max(t[3] for t in H.hpvm_batch_plan(M, N, K, 2)[1]) + 1
    g2 = max(t[3] for t in H.hpvm_batch_plan(M, N, K, 6)[1]) + 1
    assert g2 <= max(1, g1 // 2)
    # the in-leaf conversion's policies schedule as the pair policies do
    assert H.hpvm_batch_plan(M, N, K, 10) == H.hpvm_batch_plan(M, N, K, 6)
    # 256-row tiles: no tile starts at an odd multiple of 128 rows
    assert all(t[1] % 256 == 0 for t in H.hpvm_batch_plan(M, N, K, 6)[1] if t[0] >= 0)


def test_batched_workload_plan():
    shapes = W.batched_shapes()  # 512 instances, M, N, K log-uniform in [32, 2048]
    assert len(shapes) == 512
    assert all(32 <= x <= 2048 for s in shapes for x in s)
    M, N, K = zip(*shapes)
    _, slots = H.hpvm_batch_plan(M, N, K, 2)
    tiles = [t for t in slots if t[0] >= 0]
    assert len(tiles) == sum(len(_grid(m, n, b)) for (m, n, _), b in zip(shapes, H.hpvm_batch_plan(M, N, K, 2)[0]))


def test_bad_policy_and_shapes():
    with pytest.raises(H.HpvmError):
        H.hpvm_batch_plan([1], [1], [1], 12)
    with pytest.raises(H.HpvmError):
        H.hpvm_batch_plan([-1], [1], [1], 0)
