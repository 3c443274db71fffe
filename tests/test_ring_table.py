"""The ring the full pass of the inner solve follows (host table, no GPU).

Sec. 2's modulus order on the 2b columns of a pivot block pairs a with c - a
(mod 2b) at residue c; from one step to the next each pair keeps one of its
rows and takes the row that leaves the previous pair, so the b pairs form a
ring of slots.  The ring kernel relies on the table for every row it moves
and every buffer it reads, so this replays its data movement on the host:
pools of 2P + 1 row buffers per CTA, the one row a CTA sends per step, and
the CTA that forms each pair's rotation (the one holding row lo).  Any wrong
index makes a buffer hold the wrong row here."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def api():
    from paper_1008_1371_gb300 import api, build_lib

    build_lib.build()
    return api


def _cluster(b):
    return 4 if b == 16 else 8


@pytest.mark.parametrize("b", [16, 32, 64])
def test_ring_steps_are_the_modulus_steps(api, orc, b):
    """As sets, the pairs of every step are the oracle's Alg. 4.4 pairs of that
    step on 2b indices (the stepper written independently of the library)."""
    nn = 2 * b
    tab = api.hsvd_ring_table(b)
    ref = orc.modulus_pairs(nn, nn)
    assert tab.shape == (nn, b, 4)
    for s in range(nn):
        got = {(int(e[0]), int(e[1])) for e in tab[s]}
        want = {tuple(sorted(map(int, p))) for p in ref[s]}
        assert got == want, s
        assert all(e[0] < e[1] for e in tab[s])
        # every column once per step
        cols = sorted(int(x) for e in tab[s] for x in e[:2])
        assert cols == list(range(nn))


@pytest.mark.parametrize("b", [16, 32, 64])
def test_ring_moves_one_row_per_slot(api, b):
    """From step s - 1 to s slot k keeps one row and receives the other from
    slot k - 1 (cyclically); the flag names the row that moved."""
    nn, tab = 2 * b, api.hsvd_ring_table(b)
    for s in range(1, nn):
        for k in range(b):
            lo, hi, _, lo_arr = (int(x) for x in tab[s, k])
            prev, left = set(tab[s - 1, k, :2].tolist()), set(tab[s - 1, (k - 1) % b, :2].tolist())
            moved, stayed = (lo, hi) if lo_arr else (hi, lo)
            assert stayed in prev and moved in left, (s, k)
    assert not tab[0, :, 3].any()


@pytest.mark.parametrize("b", [16, 32, 64])
def test_ring_kernel_data_movement_replayed(api, b):
    """Replays k_solve_ring's row traffic: pools of 2P + 1 buffers per CTA hold
    row ids; at each step end every CTA copies the row leaving its last slot
    into the buffer the table names in the next CTA (which must be free there)
    and moves nothing else.  Then every owned slot finds rows lo and hi in the
    buffers of its table entry, each buffer in use is distinct, and every pair
    of the next step is formed exactly once, by a CTA whose pool holds row lo
    in the buffer the kernel reads (plain and look-ahead paths)."""
    nn, C = 2 * b, _cluster(b)
    P = b // C
    tab = api.hsvd_ring_table(b)
    bl = lambda e: int(e[2]) & 0xFF
    bh = lambda e: (int(e[2]) >> 8) & 0xFF
    pools = [[None] * (2 * P + 1) for _ in range(C)]
    for r in range(C):
        for kl in range(P):
            e = tab[0, r * P + kl]
            pools[r][bl(e)] = int(e[0])
            pools[r][bh(e)] = int(e[1])
    for s in range(nn):
        cur = tab[s]
        for r in range(C):
            used = []
            for kl in range(P):
                e = cur[r * P + kl]
                assert pools[r][bl(e)] == e[0] and pools[r][bh(e)] == e[1], (s, r, kl)
                used += [bl(e), bh(e)]
            assert len(set(used)) == 2 * P and max(used) <= 2 * P
        if s + 1 == nn:
            break
        nxt = tab[s + 1]
        # the pairs of step s + 1: who forms them and from which buffer
        formed = {}
        for r in range(C):
            k0 = r * P
            for l in range(P + 1):
                k = (k0 + l) % b
                e = nxt[k]
                lo_arr = bool(e[3] & 1)
                mine = (not (lo_arr and l == 0)) if l < P else lo_arr
                if not mine:
                    continue
                # plain path: row lo where it is at step s
                f = cur[(k - 1) % b if lo_arr else k]
                bf = bl(f) if f[0] == e[0] else bh(f)
                assert pools[r][bf] == e[0], (s, r, l)
                # look-ahead path: pair i holds row lo, pair j holds row hi, and pair i is this CTA's
                si = (k - 1) % b if lo_arr else k
                sj = k if lo_arr else (k - 1) % b
                fi, fj = cur[si], cur[sj]
                assert e[0] in fi[:2] and e[1] in fj[:2] and si != sj
                assert si // P == r
                assert pools[r][bl(fi)] == fi[0] and pools[r][bh(fi)] == fi[1]
                assert k not in formed, (s, k)
                formed[k] = r
        assert sorted(formed) == list(range(b))
        # the one copy per CTA, then the table's step s + 1 placement must hold
        sends = []
        for r in range(C):
            k0 = r * P
            en = nxt[(k0 + P) % b]
            lo_arr = bool(en[3] & 1)
            mv = int(en[0]) if lo_arr else int(en[1])
            dbf = bl(en) if lo_arr else bh(en)
            el = cur[k0 + P - 1]
            sbf = bl(el) if el[0] == mv else bh(el)
            assert pools[r][sbf] == mv
            sends.append(((r + 1) % C, dbf, mv, r, sbf))
        for dst, dbf, mv, src, sbf in sends:
            in_use = {x for kl in range(P) for x in (bl(cur[dst * P + kl]), bh(cur[dst * P + kl]))}
            assert dbf not in in_use, (s, dst, dbf)  # the receiving buffer is free during step s
            pools[dst][dbf] = mv
        for dst, dbf, mv, src, sbf in sends:
            if pools[src][sbf] == mv and not any(d == src and db == sbf for d, db, _, _, _ in sends):
                pools[src][sbf] = None  # the sent row's buffer is free from step s + 1


def test_ring_table_arguments(api):
    import ctypes

    out = np.zeros(8 * 64 * 64, dtype=np.int32)
    L = api.lib()
    for b in (0, 8, 48, 128):
        assert L.hsvd_ring_table(b, out.ctypes.data_as(ctypes.c_void_p)) == api.HSVD_ERR_ARG
    assert L.hsvd_ring_table(32, None) == api.HSVD_ERR_ARG
