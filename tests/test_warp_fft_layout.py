"""Host-side checks of the warp Stockham FFT's shared-memory layout (ccmf_fft.cuh).

The kernels address every radix pass as a per-lane base plus compile-time offsets: butterfly
j = lane + 32 b of the pass at sub-transform length Ns reads elements j + r N/R and writes
od + r Ns, od = (j - j mod Ns) R + j mod Ns, at padded positions wpad(i) = i + i / 16. These
tests re-derive the kernels' offset formulas and check them against wpad of the plain index for
every lane, butterfly and radix of the lengths the warp engine takes (128 ... 1024), plus the
per-pass twiddle table and the register hand-off between two transforms, and run the passes in
numpy with those index formulas to check that they compute the DFT."""

import numpy as np


def wpad(i):
    return i + (i >> 4)


def cpad(k):
    assert k % 16 == 0
    return k + k // 16


def radix(n, ns):
    rem = n // ns
    return 8 if (rem % 8 == 0 and n // 8 >= 32) else 4 if (rem % 4 == 0 and n // 4 >= 32) else 2


def passes(n):
    out, ns = [], 1
    while ns < n:
        r = radix(n, ns)
        out.append((ns, r))
        ns *= r
    return out


LENGTHS = (128, 256, 512, 1024)


def test_radix_schedule_covers_the_line():
    for n in LENGTHS:
        prod = 1
        for ns, r in passes(n):
            assert ns == prod and (n // r) % 32 == 0   # every lane takes whole butterflies
            prod *= r
        assert prod == n


def test_load_and_store_offsets_split_into_lane_base_and_constant():
    for n in LENGTHS:
        for ns, r in passes(n):
            nb = n // r
            for lane in range(32):
                if ns == 1:
                    store_base = wpad(lane * r)
                elif ns < 32:
                    jm = lane & (ns - 1)
                    store_base = wpad((lane - jm) * r + jm)
                else:
                    store_base = wpad(lane)
                for b in range(nb // 32):
                    j = lane + 32 * b
                    jm = j & (ns - 1)
                    od = (j - jm) * r + jm
                    for q in range(r):
                        assert wpad(j + q * nb) == wpad(lane) + cpad(32 * b + q * nb)
                        if ns == 1:
                            off = cpad(32 * b * r) + q
                        elif ns < 16:
                            assert ns * r >= 16
                            off = cpad(32 * b * r) + q * ns + (q * ns) // 16
                        elif ns < 32:
                            off = cpad(32 * b * r) + cpad(q * ns)
                        else:
                            kb = ((32 * b) & ~(ns - 1)) * r + ((32 * b) & (ns - 1))
                            off = cpad(kb + q * ns)
                        assert store_base + off == wpad(od + q * ns), (n, ns, lane, b, q)


def test_per_pass_twiddle_table():
    for n in LENGTHS:
        off = 0
        for ns, r in passes(n):
            if ns == 1:
                continue
            tws = n // (ns * r)
            table = {}
            for q in range((r - 1) * ns):   # the fill loop: entry q -> exponent j r tws
                table[off + q] = (q % ns) * (1 + q // ns) * tws
            for lane in range(32):
                for b in range(n // r // 32):
                    j = lane + 32 * b
                    jm = j & (ns - 1)
                    base = off + ((lane & (ns - 1)) if ns <= 32 else lane)
                    jb = 0 if ns <= 32 else ((32 * b) & (ns - 1))
                    for q in range(1, r):
                        assert table[base + jb + (q - 1) * ns] == jm * q * tws < n
            off += (r - 1) * ns
        assert off <= n   # the table fits the N entries the kernels reserve


def test_register_handoff_between_transforms():
    """The last pass (Ns >= 32) leaves lane l with elements l + 32 k in register k; the first pass
    of the next transform reads exactly those elements from the same registers."""
    for n in LENGTHS:
        ns, r = passes(n)[-1]
        assert ns >= 32
        r0 = passes(n)[0][1]
        nb0 = n // r0
        for lane in range(32):
            held = {}
            for b in range(n // r // 32):
                for q in range(r):
                    kb = ((32 * b) & ~(ns - 1)) * r + ((32 * b) & (ns - 1))
                    m = lane + kb + q * ns
                    assert (m - lane) % 32 == 0
                    held[(m - lane) // 32] = m
            assert sorted(held) == list(range(n // 32))
            for b in range(nb0 // 32):
                for q in range(r0):
                    m = lane + 32 * b + q * nb0
                    assert held[(32 * b + q * nb0) // 32] == m


def test_half_warp_bank_groups():
    """8-byte elements in half-warp groups of 16 lanes (bank pair = position mod 16): every pass's
    loads are conflict-free (2 wavefronts per warp access). The stores are too, except those of the
    second pass: 2-way conflicted at Ns = 8 (N = 256 ... 1024) and 4-way at Ns = 4 (N = 128). The GB300
    capture of the y pass at N = 512 counts the 2-way conflicts (35 extra wavefronts per line)."""
    def wavefronts(addrs):
        tot = 0
        for h in (range(16), range(16, 32)):
            groups = {}
            for lane in h:
                groups.setdefault(addrs[lane] % 16, set()).add(addrs[lane])
            tot += max(len(v) for v in groups.values())
        return tot
    for n in LENGTHS:
        for ns, r in passes(n):
            nb = n // r
            for b in range(nb // 32):
                for q in range(r):
                    loads = [wpad(lane + 32 * b + q * nb) for lane in range(32)]
                    stores = []
                    for lane in range(32):
                        j = lane + 32 * b
                        jm = j & (ns - 1)
                        stores.append(wpad((j - jm) * r + jm + q * ns))
                    assert wavefronts(loads) == 2
                    expect = {8: 4, 4: 8}.get(ns, 2)
                    assert wavefronts(stores) == expect, (n, ns, q)


def _twiddle_table(n):
    """The per-pass table as the kernels fill it: entry OFF + q of the pass at Ns holds
    W_N^{(q mod Ns)(1 + q div Ns) N / (Ns R)}, W_N = exp(-2 pi i / N)."""
    table = {}
    off = 0
    for ns, r in passes(n):
        if ns == 1:
            continue
        tws = n // (ns * r)
        for q in range((r - 1) * ns):
            table[off + q] = (q % ns) * (1 + q // ns) * tws
        off += (r - 1) * ns
    return {k: np.exp(-2j * np.pi * e / n) for k, e in table.items()}


def test_stockham_passes_compute_the_dft():
    """Run the warp Stockham passes in numpy with the kernels' index formulas (lane, butterfly,
    radix, per-pass twiddle lookups); the result is the DFT of the input line."""
    rng = np.random.default_rng(5)
    for n in LENGTHS:
        tw = _twiddle_table(n)
        x0 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        x = x0.copy()
        off = 0
        for ns, r in passes(n):
            nb = n // r
            out = np.empty_like(x)
            for lane in range(32):
                for b in range(nb // 32):
                    j = lane + 32 * b
                    vals = np.array([x[j + q * nb] for q in range(r)])
                    if ns > 1:
                        base = off + ((lane & (ns - 1)) if ns <= 32 else lane)
                        jb = 0 if ns <= 32 else ((32 * b) & (ns - 1))
                        for q in range(1, r):
                            vals[q] *= tw[base + jb + (q - 1) * ns]
                    vals = np.fft.fft(vals)   # the radix-R butterfly, forward kernel
                    jm = j & (ns - 1)
                    od = (j - jm) * r + jm
                    for q in range(r):
                        out[od + q * ns] = vals[q]
            x = out
            if ns > 1:
                off += (r - 1) * ns
        np.testing.assert_allclose(x, np.fft.fft(x0), rtol=0, atol=1e-9 * np.sqrt(n))
