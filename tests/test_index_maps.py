"""CPU models of the cluster-pair kernel's index maps (compute-sanitizer is not available on the GPU
pool, so the address arithmetic is checked here): every load, exchange and store address stays in
its shared-memory buffer, 16-byte copies are aligned, each shell element is loaded and stored
exactly once across the pair, the phi-pass slots of a ring pair are a bijection onto that pair's
memory, and the scratch blocks never overlap the CTA's own rows. Mirrors shell_kernel.cuh."""
import pytest


def swz(u, full8):
    return (u ^ ((u >> 3) & 7)) if u < full8 else u


class Pair:
    def __init__(self, Nth, Nph):
        self.Nth, self.Nph = Nth, Nph
        self.QB = Nph // 4
        self.ldc = Nph // 2 + 2
        self.q = Nth // 4
        self.A = Nth * self.ldc
        self.B = (Nth // 2) * self.ldc

    def mine(self, c, r):
        blk = c // self.QB
        lc = (c - blk * self.QB) + (self.QB if blk >= 2 else 0)
        return blk in (r, 2 + r), lc

    def brow(self, j, r):
        q = self.q
        return j - q * r if j < self.Nth // 2 else q + (j - (self.Nth - (r + 1) * q))

    def own(self, j, r):
        q, N = self.q, self.Nth
        return q * r <= j < q * (r + 1) or N - (r + 1) * q <= j < N - r * q

    def row_of(self, jr, r, fwd):
        q = self.q
        if fwd:
            return jr
        return r * q + jr if jr < q else self.Nth - (r + 1) * q + (jr - q)


SHAPES = [(128, 256), (96, 192), (8, 16), (16, 64), (64, 32)]


@pytest.mark.parametrize("Nth,Nph", SHAPES)
@pytest.mark.parametrize("fwd", [True, False])
def test_load_store_exchange(Nth, Nph, fwd):
    P = Pair(Nth, Nph)
    loaded, stored = {}, {}
    for r in (0, 1):
        rows = Nth if fwd else Nth // 2
        cols = Nph // 2 if fwd else Nph
        for jr in range(rows):
            j = P.row_of(jr, r, fwd)
            for cc in range(cols):
                c = cc if not fwd else (r * P.QB + cc if cc < P.QB else (2 + r) * P.QB + (cc - P.QB))
                m, lc = P.mine(c, r)
                if m:
                    a = j * P.ldc + lc
                    assert 0 <= a < P.A
                else:
                    assert P.own(j, r)
                    a = P.brow(j, r) * P.ldc + lc
                    assert 0 <= P.brow(j, r) < Nth // 2 and 0 <= a < P.B
                if cc % 2 == 0:
                    assert a % 2 == 0  # 16-byte cp.async pieces
                loaded.setdefault((j, c), []).append(r)
        store_rows = Nth // 2 if fwd else Nth
        for jr in range(store_rows):
            j = P.row_of(jr, r, not fwd)
            for c in range(Nph):
                m, lc = P.mine(c, r)
                if not fwd and not m:
                    continue
                if m:
                    assert 0 <= j * P.ldc + lc < P.A
                else:
                    assert P.own(j, r) and 0 <= P.brow(j, r) * P.ldc + lc < P.B
                stored.setdefault((j, c), []).append(r)
        half = Nph // 2
        for e in range((Nth // 2) * (half // 2)):
            jr, c2 = divmod(e, half // 2)
            c2 *= 2
            if fwd:
                j = P.row_of(jr, r, False)
                src, dst = j * P.ldc + c2, P.brow(j, r) * P.ldc + c2
                assert src + 1 < P.A and dst + 1 < P.B
            else:
                ro = 1 - r
                j = P.row_of(jr, ro, False)
                assert P.own(j, ro)
                src, dst = P.brow(j, ro) * P.ldc + c2, j * P.ldc + c2
                assert src + 1 < P.B and dst + 1 < P.A
            assert src % 2 == 0 and dst % 2 == 0
    assert len(loaded) == Nth * Nph and all(len(v) == 1 for v in loaded.values())
    assert len(stored) == Nth * Nph and all(len(v) == 1 for v in stored.values())


@pytest.mark.parametrize("Nth,Nph", SHAPES)
def test_phi_split_slots_are_a_bijection(Nth, Nph):
    P = Pair(Nth, Nph)
    QB8 = P.QB & ~7
    for r in (0, 1):
        for j1 in range(P.q * r, P.q * (r + 1)):
            j2 = Nth - 1 - j1
            slots = set()
            for n in range(Nph):
                seg, u = divmod(n, P.QB)
                j = j1 if seg < 2 else j2
                col = 2 * swz(u, QB8)
                a = ("B", P.brow(j, r) * P.ldc + col) if seg & 1 else ("A", j * P.ldc + col)
                slots |= {a, (a[0], a[1] + 1)}
            elems = set()
            for k in range(Nph):
                for j in (j1, j2):
                    m, lc = P.mine(k, r)
                    elems.add(("A", j * P.ldc + lc) if m else ("B", P.brow(j, r) * P.ldc + lc))
            assert slots == elems and len(slots) == 2 * Nph


@pytest.mark.parametrize("Nth,Nph", SHAPES)
def test_scratch_blocks_are_free_memory(Nth, Nph):
    P = Pair(Nth, Nph)
    q = P.q
    cap_ph = (q * P.ldc * 8) // (16 * Nph)
    cap_th = (8 * (Nth // 2) * P.ldc) // (16 * 2 * Nth)
    if cap_ph < 1 or cap_th < 1:
        pytest.skip("the plan does not choose the cluster kernel for this shape (no scratch room)")
    assert cap_th * 2 * Nth * 16 <= P.B * 8  # theta scratch fits buffer B
    for r in (0, 1):
        ro = 1 - r
        blocks = [(q * ro, q * ro + q), (Nth - (ro + 1) * q, Nth - ro * q)]
        for lo, hi in blocks:
            assert not any(P.own(j, r) for j in range(lo, hi))  # the peer's rows only
            assert (lo * P.ldc * 8) % 16 == 0
            assert lo * P.ldc * 8 + cap_ph * Nph * 16 <= hi * P.ldc * 8


@pytest.mark.parametrize("n", [8, 16, 24, 64, 100, 128])
def test_swizzle_is_a_permutation_and_spreads_strides(n):
    full8 = n & ~7
    assert sorted(swz(u, full8) for u in range(n)) == list(range(n))
    # 8 consecutive 16-byte slots at stride 1, 2, 4 or 8 land on 8 different bank groups
    for stride in (1, 2, 4, 8):
        for start in range(0, full8 - 7 * stride, 8):
            groups = {swz(start + t * stride, full8) % 8 for t in range(8)}
            assert len(groups) == 8, (stride, start)
