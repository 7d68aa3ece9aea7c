"""The arithmetic the large-precision tensor engine (p = 4096 .. 32768) relies
on, checked exactly with Python integers on the CPU: 8-bit balanced digits of
the multiplier against 4-bit balanced digits of the pivot-row element, the
radix-16 column sums and their bound (exact in fp32 with the magic bias for
every n <= 1024), the limb formula of the epilogue on raw fp32 words, the
lazy low half (when the band of limbs n-32 .. n-2 holds both a one and a zero,
the upper limbs, limb n-1 and a non-zero sticky bit follow from the formed
positions alone), the tiles' K ranges (every non-zero term of a tile inside
its MMA K steps) and the core addressing of the B operand (d = n-core +
2 k-core), and the MMA work count bench.py reports.  Small n, the same
formulas."""
import random

import numpy as np
import pytest

import bench


def balanced(m, nd, bits):
    """Digits in [-2^(bits-1), 2^(bits-1)) and the carry out of the top."""
    R, h = 1 << bits, 1 << (bits - 1)
    d, c = [], 0
    for s in range(nd):
        v = ((m >> (bits * s)) & (R - 1)) + c
        c = 1 if v >= h else 0
        d.append(v - R * c)
    return d, c


def product_sums(n, z, b):
    KD, KB = 4 * n, 8 * n
    e, cz = balanced(z, KD, 8)
    f, cb = balanced(b, KB, 4)
    fb = f + [1]
    c = [0] * (16 * n)
    for s in range(KD):
        if e[s]:
            for t in range(KB + 1):
                c[2 * s + t] += e[s] * fb[t]
    return e, cz, f, cb, c


def tiles(n):
    KD, KB, R0, T = 4 * n, 8 * n, 8 * n - 256, n // 32 + 1
    out = []
    for tau in range(T):
        rho = R0 + 256 * tau
        lo = (KD - 1 - min((rho + 255) // 2, KD - 1)) // 16
        hi = (KD - 1 - ((rho - KB + 1) // 2 if rho > KB else 0)) // 16 + 1
        out.append((rho, lo, hi))
    return out


def epilogue(n, c, b):
    """Limbs from the formed positions (r >= R0) with the raw-fp32-word
    formula, carry-in zero, 2^p b added from limb n on."""
    KD, R0 = 4 * n, 8 * n - 256
    kOff = 1016 * KD
    magic = np.float32(2 ** 23 + kOff)
    acc, limbs = 0, {}
    for r0 in range(R0, 16 * n, 8):
        w = [int((np.float32(c[r0 + q]) + magic).view(np.uint32)) for q in range(8)]
        a = [(w[2 * k] + (w[2 * k + 1] << 4) + 0x05000000) & 0xFFFFFFFF for k in range(4)]
        acc += a[0] + (a[1] << 8) + (a[2] << 16) + (a[3] << 24) - kOff * 0x11111111
        L = r0 // 8
        if L >= n:
            acc += (b >> (32 * (L - n))) & 0xFFFFFFFF
        limbs[L] = acc & 0xFFFFFFFF
        acc >>= 32
    return limbs, acc


def band_decides(n, limbs):
    l0 = limbs[n - 32]
    mid = [limbs[L] for L in range(n - 31, n - 1)]
    orv, andv = 0, 0xFFFFFFFF
    for v in mid:
        orv |= v
        andv &= v
    return ((l0 >> 19) | orv) != 0 and (((~l0 & 0xFFFFFFFF) >> 19) | (andv ^ 0xFFFFFFFF)) != 0


@pytest.mark.parametrize("n", [32, 64, 128])
def test_digits_sums_and_epilogue(n):
    p, KD = 32 * n, 4 * n
    g = random.Random(4000 + n)
    cases = [(g.getrandbits(p) | (1 << (p - 1)), g.getrandbits(p) | (1 << (p - 1))) for _ in range(3)]
    cases += [((1 << p) - 1, (1 << p) - 1), (1 << (p - 1), (1 << p) - 1),
              (int("80" * (p // 8), 16), int("8" * (p // 4), 16)), (int("ff80" * (p // 16), 16), int("f8" * (p // 8), 16))]
    decided = 0
    for z, b in cases:
        e, cz, f, cb, c = product_sums(n, z, b)
        assert cz == 1 and cb == 1  # normalised mantissas carry out of the top digit
        assert sum(v << (8 * s) for s, v in enumerate(e)) + (1 << p) == z
        assert sum(v << (4 * t) for t, v in enumerate(f)) + (1 << p) == b
        # the nibbles are those of b + 0x88..8, less 8
        t8 = b + int("8" * (8 * n), 16)
        assert [((t8 >> (4 * i)) & 15) - 8 for i in range(8 * n)] == f
        assert all(-1016 * KD <= v <= 1024 * KD for v in c)
        P = sum(v << (4 * r) for r, v in enumerate(c)) + (b << p)
        assert P == z * b
        limbs, top = epilogue(n, c, b)
        if band_decides(n, limbs):
            decided += 1
            assert top == 0
            for L in range(n - 1, 2 * n):
                assert limbs[L] == (P >> (32 * L)) & 0xFFFFFFFF
            assert P & ((1 << (32 * (n - 1))) - 1) != 0  # the sticky bit is 1
    assert decided >= 3  # the random operands take the formed positions alone


def test_window_fits_fp32_at_every_precision():
    for n in (128, 256, 512, 1024):
        KD = 4 * n
        lo, hi = -1016 * KD, 1024 * KD
        assert hi - lo < 2 ** 23  # [2^23, 2^24) holds the biased window
        magic = 2 ** 23 + 1016 * KD
        assert float(np.float32(magic)) == magic
        # both bias constants are exact in bf16 (8 significant bits)
        for v in (2 ** 23, 1016 * KD):
            f = np.array([v], np.float32)
            assert (f.view(np.uint32) & 0xFFFF)[0] == 0


@pytest.mark.parametrize("n", [32, 64, 128])
def test_tile_k_ranges_cover_every_term(n):
    KD, KB = 4 * n, 8 * n
    g = random.Random(n)
    p = 32 * n
    e, _, f, _, _ = product_sums(n, g.getrandbits(p) | (1 << (p - 1)), g.getrandbits(p) | (1 << (p - 1)))
    fb = f + [1]
    for rho, lo, hi in tiles(n):
        for r in range(rho, rho + 256):
            for s in range(KD):
                t = r - 2 * s
                if 0 <= t <= KB and e[s] and fb[t]:
                    assert lo * 16 <= KD - 1 - s < hi * 16


def test_b_core_addressing():
    """Element (k', r) of the B operand at the descriptor address (leading
    offset 256, stride offset 128, start 128 (32 t + 4 (ks - KSPS sg)) in the
    stage window of cores d0 .. d0 + NCORE - 1, d0 = n-core(R0 + 512 pi) +
    4 KSPS sg; KSPS = 16 MMA K steps per stage, NCORE = 128) holds
    f~(r - 2 s) with s = KD - 1 - k'."""
    n, KSPS, NCORE = 64, 16, 128
    KD, KB, R0 = 4 * n, 8 * n, 8 * n - 256
    g = random.Random(5)
    f, _ = balanced(g.getrandbits(32 * n) | (1 << (32 * n - 1)), KB, 4)
    fb = f + [1]

    def ft(x):
        return fb[x] if 0 <= x <= KB else 0

    T = n // 32 + 1
    for pi in range((T + 1) // 2):
        nc0 = (R0 + 512 * pi) // 8
        for sg in range(KD // (16 * KSPS)):
            d0 = nc0 + 4 * KSPS * sg
            core = {}
            for dl in range(NCORE):
                for rr in range(8):
                    for kk in range(8):
                        core[dl * 128 + rr * 16 + kk * 2] = ft(8 * (d0 + dl) + rr + 2 * kk - 2 * KD + 2)
            for t in range(2 if 2 * pi + 1 < T else 1):
                for ks in range(KSPS * sg, KSPS * sg + KSPS):
                    start = 128 * (32 * t + 4 * (ks - KSPS * sg))
                    for kl in range(16):
                        for nn in range(0, 256, 13):
                            addr = start + (nn // 8) * 128 + (kl // 8) * 256 + (nn % 8) * 16 + (kl % 8) * 2
                            assert addr < NCORE * 128
                            r = R0 + 512 * pi + 256 * t + nn
                            s = KD - 1 - (16 * ks + kl)
                            assert core[addr] == ft(r - 2 * s)


@pytest.mark.parametrize("n", [128, 1024])
def test_mma_work_count(n):
    """bench.tcl_mma_macs_per_product: the K steps the engine issues per tile,
    times 16 x 256 MACs; at most the schoolbook 8 x 4-bit count 32 n^2."""
    want = sum((hi - lo) * 16 * 256 for _, lo, hi in tiles(n))
    assert bench.tcl_mma_macs_per_product(32 * n) == want
    assert want <= 32 * n * n


def stage_plan(n, KSPS):
    """The stages of one column: (pass, stage index sg, [(tile t, first K
    step, end K step)]) in issue order, from the tiles' K ranges."""
    T = n // 32 + 1
    tl = tiles(n)
    plan = []
    for pi in range((T + 1) // 2):
        ts = [t for t in range(2) if 2 * pi + t < T]
        lo = min(tl[2 * pi + t][1] for t in ts) // KSPS
        hi = (max(tl[2 * pi + t][2] for t in ts) + KSPS - 1) // KSPS
        for sg in range(lo, hi):
            work = []
            for t in ts:
                a = max(tl[2 * pi + t][1], KSPS * sg)
                b = min(tl[2 * pi + t][2], KSPS * sg + KSPS)
                if a < b:
                    work.append((t, a, b))
            plan.append((pi, sg, sg == lo, sg + 1 == hi, work))
    return plan


@pytest.mark.parametrize("n,KSPS,STAGES", [(128, 16, 2), (256, 16, 2), (1024, 16, 2), (128, 8, 3), (512, 4, 4)])
def test_b_core_ring(n, KSPS, STAGES):
    """The sliding ring of B cores: NCORE = 63 + 4 KSPS rounded up to 16
    cores per window, RING = STAGES NCORE slots plus a mirror of the first
    NCORE - 4 KSPS.  The builders of a stage write its new cores (all of the
    window at a pass's first stage, else the last 4 KSPS) at the window start
    + dl, mirrored below MIRROR; the window start advances by 4 KSPS per stage
    and NCORE after a pass's last one.  Every core an MMA of the stage reads
    (start 32 t + 4 kl, 32 n-cores at stride 1, 2 k-cores at stride 2) holds
    core d = n-core + 2 k-core, and it still does while the next STAGES - 1
    stages are built (the builders of stage g wait only for stage g - STAGES).
    Two columns, so the ring wraps across items."""
    NCORE = (63 + 4 * KSPS + 15) // 16 * 16
    assert NCORE % (4 * KSPS) == 0
    RING, MIRROR = STAGES * NCORE, NCORE - 4 * KSPS
    R0 = 8 * n - 256
    ring = [None] * (RING + MIRROR)
    plan = stage_plan(n, KSPS) * 2
    wb = wm = 0
    inflight = []  # (window start, expected cores by slot offset) of stages not yet complete
    for g, (pi, sg, first, last, work) in enumerate(plan):
        nc0 = (R0 + 512 * pi) // 8
        d0 = nc0 + 4 * KSPS * sg
        for dl in range(0 if first else NCORE - 4 * KSPS, NCORE):
            x = wb + dl
            if x >= RING:
                x -= RING
            ring[x] = d0 + dl
            if x < MIRROR:
                ring[x + RING] = d0 + dl
        wb += NCORE if last else 4 * KSPS
        if wb >= RING:
            wb -= RING
        reads = {}
        for t, a, b in work:
            for ks in range(a, b):
                kl = ks - KSPS * sg
                for c in range(32):
                    for kc in range(2):
                        dl = 32 * t + 4 * kl + c + 2 * kc
                        ncore = (R0 + 512 * pi + 256 * t) // 8 + c
                        kcore = 2 * ks + kc
                        reads[dl] = ncore + 2 * kcore
        assert max(reads) < NCORE
        inflight.append((wm, reads))
        inflight = inflight[-STAGES:]  # stage g - STAGES has completed
        for w, rd in inflight:
            assert w + max(rd) < RING + MIRROR
            for dl, d in rd.items():
                assert ring[w + dl] == d, (g, dl)
        wm += NCORE if last else 4 * KSPS
        if wm >= RING:
            wm -= RING
        assert wm % (4 * KSPS) == 0


@pytest.mark.parametrize("n", [128, 1024])
def test_epilogue_b_limbs_by_pass(n):
    """The epilogue's b limbs: pass pi's 64 limbs L = n - 32 + 64 pi + o
    (o = 0..63) need b's limb L - n (zero below limb n).  Lane l loads offsets
    l and 32 + l (b[64 pi - 32 + l], b[64 pi + l], zero outside [0, n)); chunk
    ch takes limb l4 from lane (4 ch + l4) mod 32 of word ch >= 8."""
    g = random.Random(n)
    b = [g.getrandbits(32) for _ in range(n)]
    T = n // 32 + 1
    for pi in range((T + 1) // 2):
        w0 = [b[64 * pi - 32 + l] if 0 <= 64 * pi - 32 + l < n else 0 for l in range(32)]
        w1 = [b[64 * pi + l] if 64 * pi + l < n else 0 for l in range(32)]
        nch = 16 if 2 * pi + 1 < T else 8
        for ch in range(nch):
            src = w1 if ch >= 8 else w0
            for l4 in range(4):
                L = n - 32 + 64 * pi + 4 * ch + l4
                assert L < 2 * n
                want = b[L - n] if L >= n else 0
                assert src[(4 * ch + l4) % 32] == want
