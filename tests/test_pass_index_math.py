"""Host-side checks of the pass kernels' index arithmetic (no GPU): the pass plans and the
tile -> amplitude mappings of the one-tile, pipelined and cluster-pair kernels, re-derived
from their definitions (csrc/uapply.cu make_plan, csrc/pass_kernel.cuh, pass_pipe.cuh,
pass_pair.cuh). Every amplitude must belong to exactly one tile position of each pass, every
qubit must be kicked exactly once per U application, and the padded shared-memory positions
must be a per-thread base plus a per-register constant inside the buffer.
"""

import pytest


def make_plan(L, nb, min_cols):
    """(NB, c, start, kick_from) per pass: the first kicks qubits [0, NB) in contiguous
    tiles, each later one keeps >= min_cols low column bits and kicks the next qubits."""
    if L <= nb:
        return [(L, L, L, 0)]
    plan = [(nb, nb, nb, 0)]
    q0 = nb
    while q0 < L:
        nq = min(L - q0, nb - min_cols)
        c = nb - nq
        plan.append((nb, c, q0, c))
        q0 += nq
    return plan


def kicked_qubits(plan):
    out = []
    for (nb, c, start, kf) in plan:
        if kf == 0:
            out += list(range(nb))
        else:
            out += list(range(start, start + nb - c))
    return sorted(out)


def tile_indices(L, nb, c, start, RB, tile):
    """Global indices the kernel touches for one tile: thread t, register r -> tile element
    t | (r << g_top) -> bits [0, c) + ((e >> c) << start) + CTA base."""
    single = nb == L
    midbits = 0 if single else start - c
    topshift = L if single else start + nb - c
    mid = tile & ((1 << midbits) - 1)
    top = tile >> midbits
    base = (mid << c) | (top << topshift)
    cmask = (1 << c) - 1
    g_top = nb - RB
    f = lambda e: (e & cmask) + ((e >> c) << start)
    out = []
    for t in range(1 << (nb - RB)):
        for r in range(1 << RB):
            out.append(base + f(t) + f(r << g_top))
    return out


@pytest.mark.parametrize("nb,cols", [(12, 4), (11, 3), (11, 2), (10, 3), (10, 2), (9, 3)])
def test_plans_kick_every_qubit_once(nb, cols):
    for L in range(3, 25):
        plan = make_plan(L, nb, cols)
        assert kicked_qubits(plan) == list(range(L)), (L, plan)
        for (b, c, start, kf) in plan[1:]:
            assert c >= cols and start + b - c <= L


@pytest.mark.parametrize("nb,RB,cols", [(11, 3, 2), (10, 3, 2), (12, 4, 4), (9, 3, 3)])
def test_every_amplitude_once_per_pass(nb, RB, cols):
    for L in range(nb, 17):
        for (b, c, start, kf) in make_plan(L, nb, cols):
            rb = min(RB, b)
            hit = bytearray(1 << L)
            for tile in range(1 << (L - b)):
                for s in tile_indices(L, b, c, start, rb, tile):
                    assert 0 <= s < (1 << L)
                    hit[s] += 1
            assert min(hit) == 1 and max(hit) == 1, (L, (b, c, start))


def test_cluster_pair_halves_and_partner_bit():
    # a 2^11 tile split over two CTAs of 2^10: CTA rank q, thread t, register r address
    # base + f(t) + f(q << 10) + f(r << 7); every amplitude once, and partners (q = 0, 1 at
    # the same t, r) differ in exactly one bit: the qubit of the tile's top bit
    NBL, RB = 10, 3
    for L in range(12, 17):
        for (b, c, start, kf) in make_plan(L, NBL + 1, 2):
            single = b == L
            midbits = 0 if single else start - c
            topshift = L if single else start + b - c
            cmask = (1 << c) - 1
            f = lambda e: (e & cmask) + ((e >> c) << start)
            hit = bytearray(1 << L)
            for tile in range(1 << (L - b)):
                base = ((tile & ((1 << midbits) - 1)) << c) | ((tile >> midbits) << topshift)
                for t in range(1 << (NBL - RB)):
                    for r in range(1 << RB):
                        s0 = base + f(t) + f(r << (NBL - RB))
                        s1 = s0 + f(1 << NBL)
                        x = s0 ^ s1
                        assert x and x & (x - 1) == 0
                        hit[s0] += 1
                        hit[s1] += 1
            assert min(hit) == 1 and max(hit) == 1, (L, (b, c, start))


def _smem_pos(e, RB):
    return e + (e >> RB)


def _tile_elem(t, r, g, RB):
    return (t & ((1 << g) - 1)) | (r << g) | ((t >> g) << (g + RB))


@pytest.mark.parametrize("nb,RB", [(11, 3), (10, 3), (12, 3), (11, 2), (12, 4)])
def test_shared_memory_positions_split(nb, RB):
    # pos(t, r, g) = base_t(g) + const_r(g), distinct, inside the padded buffer
    slot = (1 << nb) + (1 << (nb - RB))
    for g in range(0, nb - RB + 1):
        seen = set()
        for t in range(1 << (nb - RB)):
            b = (t & ((1 << g) - 1)) | ((t >> g) << (g + RB))
            base = b + (b >> RB)
            for r in range(1 << RB):
                p = _smem_pos(_tile_elem(t, r, g, RB), RB)
                assert p == base + (r << g) + ((r << g) >> RB)
                assert 0 <= p < slot
                seen.add(p)
        assert len(seen) == 1 << nb


@pytest.mark.parametrize("nb,RB", [(11, 3), (10, 3), (12, 3), (11, 2)])
@pytest.mark.parametrize("kf", [0, 2, 3, 4])
def test_pipelined_rounds_kick_tile_bits_once(nb, RB, kf):
    # register rounds from the top: round 0 at g = NB - RB, transpose i to
    # max(NB - RB (i + 2), 0) while the previous round's g exceeds KF; each round kicks its
    # register bits in [KF, previous g)
    gs, hi = [nb - RB], nb - RB
    while hi > kf:
        hi = max(hi - RB, 0)
        gs.append(hi)
    his = [nb] + gs[:-1]
    kicked = [g + b for g, h in zip(gs, his) for b in range(RB) if kf <= g + b < h]
    assert sorted(kicked) == list(range(kf, nb))


def test_library_plan_matches_the_derivation():
    # the plan and the derived index shifts the library itself uses (host-only C-ABI query),
    # against the derivation above: a change to the C++ plan fails here
    from paper_2102_05054_gb300 import build, floquet
    build.build()
    for L in range(3, 25):
        for nb, cols in [(9, 3), (10, 3), (10, 4), (11, 2), (11, 3), (11, 4), (12, 3), (12, 4)]:
            got = floquet.pass_plan(L, nb, cols)
            want = make_plan(L, nb, cols)
            assert [g[:4] for g in got] == [tuple(w) for w in want], (L, nb, cols)
            for (b, c, start, kf, mid, top) in got:
                if b == L:
                    assert (mid, top) == (0, L)
                else:
                    assert (mid, top) == (start - c, start + b - c)
    with pytest.raises(RuntimeError):
        floquet.pass_plan(20, 11, 11)   # min_cols must leave qubits to kick
