"""The arithmetic the tensor engine for p = 512, 1024 and 2048 (k_update_tcp:
KD = 64, 128, 256 balanced 8-bit digits per mantissa) relies on, modelled
exactly on the CPU with Python integers and numpy float32, from the operand
bytes the kernel writes to the limbs and the rounded product it stages:

- the A operand: the multiplier's balanced digits as the bytes of
  z + 0x8080..80 less 128 (the carry out of the top is the 2^p of
  z = z' + 2^p), digit s at K position KD - 1 - s, ones at KD .. KD + 2;
- the B operand: b~ = b's balanced digits (per-lane carry lookahead over the
  ballots) and the carry digit 1, in Hankel cores (core d, row nn, element kk
  holds b~[8 d + nn + kk - KD + 1]) read through a no-swizzle descriptor with
  equal leading and stride offsets; the extra K step's raw digits of b and the
  bias constants 2^23 and kOff;
- the MMAs: only the K steps each tile needs (neighbouring tiles with the same
  range merged into one N = 256 MMA), the extra step last; every column sum
  is exact in fp32 and lies in [-4161536, 4194559];
- the epilogue: raw fp32 words (the FADD of the magic constant in the lower
  tiles, the MMA's own bias in the upper ones) into limbs by two 32-bit
  shift-adds and one multiply-add per limb, less one constant; the lazy low
  half (a carry chain from limb NL - 8 with a zero carry, the low chunks read
  only when bits [14, 224) of limbs NL - 8 .. NL - 2 are all ones or all
  zeros) and the bound that makes it exact;
- round_product: the staged upper limbs, limb NL - 1 and the sticky OR rounded
  to p bits, against round to nearest even of the exact product.

The Python model follows the kernel's formulas; the exact products and the
rounding it is checked against are plain integer arithmetic."""
import random

import numpy as np
import pytest

KDS = [64, 128, 256]  # p = 512, 1024, 2048
K_OFF = 255 * 2 ** 14  # 4177920
K_MAGIC = 2 ** 23 + K_OFF
K_C = K_OFF * 0x01010101 + 0x4B000000 * 0x10001
MASK = 0xFFFFFFFF


class Geo:
    """The kernel's geometry for mantissas of KD 8-bit digits."""

    def __init__(self, KD):
        self.KD, self.NL = KD, KD // 4
        self.TILES = 2 * KD // 128  # 128-column tensor-memory tiles
        self.NCORE = 16 * self.TILES + KD // 8 - 1  # Hankel cores
        self.XT0 = KD // 128  # first tile with positions >= KD
        self.KA = KD + 16  # A's K extent: the digits and the extra K step
        self.K0 = self.NL // 8 - 1  # first chunk of 32 sums the epilogue reads
        self.NCH = 4 * self.TILES

    def ks_lo(self, t):
        v = self.KD - 128 * (t + 1)
        return v // 16 if v > 0 else 0

    def ks_hi(self, t):
        v = 2 * self.KD - 128 * t
        return v // 16 if v < self.KD else self.KD // 16

    def merge(self, t):
        return t + 1 < self.TILES and self.ks_lo(t) == self.ks_lo(t + 1) and self.ks_hi(t) == self.ks_hi(t + 1)

    def groups(self):
        """(first tile, tiles in the MMA) in issue order."""
        out, t = [], 0
        while t < self.TILES:
            two = self.merge(t)
            out.append((t, 2 if two else 1))
            t += 2 if two else 1
        return out


def balanced(m, nd):
    """Balanced 8-bit digits in [-128, 127] and the carry out of the top."""
    d, c = [], 0
    for s in range(nd):
        v = ((m >> (8 * s)) & 255) + c
        c = 1 if v >= 128 else 0
        d.append(v - 256 * c)
    return d, c


def bf16_exact(v):
    """bf16 bits of a small integer through fp32 (the top half of the fp32
    bits); asserts nothing is cut off."""
    w = int(np.array([v], np.float32).view(np.uint32)[0])
    assert w & 0xFFFF == 0
    return w >> 16


def bf16_value(h):
    return float(np.array([h << 16], np.uint32).view(np.float32)[0])


def a_row(z, g):
    """The A row of multiplier mantissa z (K positions 0 .. KA - 1), built
    like the kernel: one carry chain adds 0x80808080 to every limb, byte q of
    limb L less 128 is digit 4 L + q at K position KD - 4 - 4 L + (3 - q); the
    extra K step has ones at KD, KD + 1, KD + 2."""
    NL, KD = g.NL, g.KD
    f, c = [], 0
    for L in range(NL):
        v = ((z >> (32 * L)) & MASK) + 0x80808080 + c
        f.append(v & MASK)
        c = v >> 32
    assert c == 1  # a normalised mantissa: the dropped carry is the 2^p
    row = [0.0] * g.KA
    for L in range(NL):
        for q in range(4):
            byte = (f[L] >> (8 * q)) & 255
            # (2^23 + byte) - (2^23 + 128) in fp32, then its top 16 bits
            x = np.float32(np.array([0x4B000000 | byte], np.uint32).view(np.float32)[0]) - np.float32(8388736.0)
            h = bf16_exact(float(x))
            assert bf16_value(h) == byte - 128
            row[KD - 1 - (4 * L + q)] = bf16_value(h)
    for k in (KD, KD + 1, KD + 2):
        row[k] = bf16_value(0x3F80)
    return row


def carry_mask(gen, prop, inject):
    """Carry into every lane (bit l) and out of lane 31 (bit 32) from the
    lanes' generate and propagate bits: (P + 2 G + c0) xor P."""
    return (prop + (gen << 1) + inject) ^ prop


def b_tilde(b, g):
    """b's balanced digits and the carry digit at KD as the builder warp forms
    them: 32 lanes of KD / 32 digits, each lane's carry out for carry-in 0 and
    1, the carry-in of every lane from one carry lookahead."""
    KD = g.KD
    DPL = KD // 32
    by = [(b >> (8 * s)) & 255 for s in range(KD)]
    gen = prop = 0
    for l in range(32):
        f0, f1 = 0, 1
        for q in range(DPL):
            d = by[l * DPL + q]
            f0 = 1 if d + f0 >= 128 else 0
            f1 = 1 if d + f1 >= 128 else 0
        gen |= f0 << l
        prop |= (1 if (f1 and not f0) else 0) << l
    cm = carry_mask(gen, prop, 0)
    out = [0] * (KD + 1)
    for l in range(32):
        cy = (cm >> l) & 1
        for q in range(DPL):
            t = by[l * DPL + q] + cy
            cy = 1 if t >= 128 else 0
            out[l * DPL + q] = t - 256 * cy
    out[KD] = (cm >> 32) & 1
    return out


def hankel_buffer(bt, g):
    """The Hankel buffer as bf16 values by element (2-byte) index: zero, then
    cores KD/8 - 1 .. KD/4 - 1 rebuilt from b~."""
    KD = g.KD
    H = np.zeros(g.NCORE * 64, np.float64)
    for q in range((KD // 8 + 1) * 8):
        d, nn = KD // 8 - 1 + (q >> 3), q & 7
        base = 8 * d + nn - (KD - 1)
        for kk in range(8):
            idx = base + kk
            v = bt[idx] if 0 <= idx <= KD else 0
            H[(d * 128 + nn * 16 + kk * 2) // 2] = bf16_value(bf16_exact(v))
    return H


def extra_buffer(b, g):
    """The extra K step's B operand (tiles XT0 ..): in k-core 0 of every
    n-core row, element 1 = 2^23 and element 2 = kOff; element 0 = b's raw
    digit r - KD at output position r."""
    XTN = g.TILES - g.XT0
    X = np.zeros(XTN * 4096 // 2, np.float64)
    for o in range(0, XTN * 4096, 16):
        if (o & 255) < 128:
            X[o // 2 + 1] = bf16_value(0x4B00)
            X[o // 2 + 2] = bf16_value(0x4A7F)
    assert bf16_value(0x4B00) == 2 ** 23 and bf16_value(0x4A7F) == K_OFF
    for r in range(128 * g.XT0, 128 * g.TILES):
        j = r - g.KD
        v = (b >> (8 * j)) & 255 if 0 <= j < g.KD else 0
        X[((r // 128 - g.XT0) * 4096 + ((r % 128) // 8) * 256 + (r % 8) * 16) // 2] = bf16_value(bf16_exact(v))
    return X


def mma_sums(A, H, X, g):
    """Column sums as the MMAs form them: per tile group the K steps
    [ks_lo, ks_hi) with B read at the descriptor's addresses (start
    (16 t + 2 ks) cores, n-core stride 128 B, k-core stride 128 B), then the
    extra K step per upper tile (n-core stride 256 B, k-core stride 128 B).
    Returns the sums and, per position, the sum of |terms| of the digit steps
    (a bound on every partial sum, whatever the accumulation order)."""
    D = np.zeros(128 * g.TILES, np.float64)
    absum = np.zeros(128 * g.TILES, np.float64)
    A = np.asarray(A)
    n = np.arange(256)[:, None]
    kl = np.arange(16)[None, :]
    for t, cnt in g.groups():
        N = 128 * cnt
        for ks in range(g.ks_lo(t), g.ks_hi(t)):
            byte = (16 * t + 2 * ks) * 128 + (n[:N] // 8) * 128 + (kl // 8) * 128 + (n[:N] % 8) * 16 + (kl % 8) * 2
            assert byte.max() < g.NCORE * 128
            Bt = H[byte // 2]  # [N, 16]
            terms = Bt * A[16 * ks: 16 * ks + 16][None, :]
            D[128 * t: 128 * t + N] += terms.sum(axis=1)
            absum[128 * t: 128 * t + N] += np.abs(terms).sum(axis=1)
    for u in range(g.XT0, g.TILES):
        byte = (u - g.XT0) * 4096 + (n[:128] // 8) * 256 + (kl // 8) * 128 + (n[:128] % 8) * 16 + (kl % 8) * 2
        Bt = X[byte // 2]
        D[128 * u: 128 * u + 128] += (Bt * A[g.KD: g.KD + 16][None, :]).sum(axis=1)
    return D, absum


def fp32_words(D, g):
    """The raw fp32 words the epilogue reads: the MMA's biased sums in the
    upper tiles, sum + kMagic by one fp32 add in the lower ones."""
    w = []
    for r, v in enumerate(D):
        if r // 128 >= g.XT0:
            assert 2 ** 23 <= v < 2 ** 24 and v == int(v)
            w.append(int(np.array([v], np.float32).view(np.uint32)[0]))
        else:
            assert abs(v) < 2 ** 23 and v == int(v)
            s = np.float32(v) + np.float32(K_MAGIC)
            w.append(int(np.array([s], np.float32).view(np.uint32)[0]))
    return w


def limbs8(w, ac):
    """Eight limbs from 32 raw words and the running carry."""
    lim = []
    for q in range(8):
        u = w[4 * q: 4 * q + 4]
        xl = (u[0] + (u[1] << 8)) & MASK
        yl = (u[2] + (u[3] << 8)) & MASK
        ac += yl * 65536 + xl - K_C
        lim.append(ac & MASK)
        ac >>= 32  # arithmetic, as int64 >> 32
    return lim, ac


def epilogue(w, g):
    """The epilogue of one row: the upper NL limbs, limb NL - 1, the sticky
    word, whether the low chunks were read, and the carry left at the end."""
    NL, K0 = g.NL, g.K0
    acc, upper, exact_path = 0, {}, False
    l63 = sticky = None
    for k in range(K0, g.NCH):
        lim, acc = limbs8(w[32 * k: 32 * k + 32], acc)
        if 8 * k >= NL:
            for q in range(8):
                upper[8 * k + q - NL] = lim[q]
            continue
        lo7 = hi7 = None
        lo7 = lim[1] | lim[2] | lim[3] | lim[4] | lim[5] | lim[6]
        hi7 = lim[1] & lim[2] & lim[3] & lim[4] & lim[5] & lim[6]
        any1 = ((lim[0] >> 14) | lo7) != 0
        any0 = (((~lim[0] & MASK) >> 14) | (~hi7 & MASK)) != 0
        l63, sticky = lim[7], 1
        if not (any1 and any0):
            exact_path = True
            ac2, slo = 0, 0
            for kk in range(K0):
                l8, ac2 = limbs8(w[32 * kk: 32 * kk + 32], ac2)
                for v in l8:
                    slo |= v
            t = ac2
            for q in range(8):
                t += lim[q]
                lim[q] = t & MASK
                t >>= 32
            acc += t
            l63 = lim[7]
            sticky = slo | lim[0] | lim[1] | lim[2] | lim[3] | lim[4] | lim[5] | lim[6]
    return [upper[i] for i in range(NL)], l63, sticky, exact_path, acc


def round_product(up, l63, sticky, NL):
    """round_product: shift a 2p - 1 bit product up one bit, round to nearest
    even with limb NL - 1 and the sticky word; returns the mantissa and the
    exponent adjustment."""
    up = list(up)
    top = up[NL - 1] >> 31
    sft = 1 - top
    if sft:
        for q in range(NL - 1, 0, -1):
            up[q] = ((up[q] << 1) | (up[q - 1] >> 31)) & MASK
        up[0] = ((up[0] << 1) | (l63 >> 31)) & MASK
    rbit = (l63 >> (31 - sft)) & 1
    st = (l63 & (0x7FFFFFFF >> sft)) | sticky
    inc = rbit & (1 if (st != 0 or (up[0] & 1)) else 0)
    m = sum(v << (32 * q) for q, v in enumerate(up)) + inc
    ovf = m >> (32 * NL)
    if ovf:
        m = 1 << (32 * NL - 1)
    return m, (0 if top else -1) + ovf


def rne_product(z, b, p):
    """Round to nearest even of z b at p bits: the mantissa and the exponent
    adjustment against e_z + e_b (0 for a 2p-bit product, -1 for 2p - 1,
    +1 more when rounding carries out)."""
    P = z * b
    sh = P.bit_length() - p
    q, r = divmod(P, 1 << sh)
    half = 1 << (sh - 1)
    if r > half or (r == half and q & 1):
        q += 1
    adj = P.bit_length() - 2 * p
    if q >> p:
        q >>= 1
        adj += 1
    return q, adj


def operands(KD, seed):
    p = 8 * KD
    g = random.Random(seed)
    top = 1 << (p - 1)
    cases = [(g.getrandbits(p) | top, g.getrandbits(p) | top) for _ in range(4)]
    cases += [
        ((1 << p) - 1, (1 << p) - 1),  # all ones
        (top, g.getrandbits(p) | top),  # a power of two: exact product, low limbs zero
        (g.getrandbits(p) | top, top),
        (top + 1, 3 << (p - 2)),  # an exact tie at bit p (2p - 1 bit product), odd: rounds up
        (top + 2, top + (1 << (p - 3))),  # an exact tie, even: stays
        (top + 1, top + (1 << (p - 2)) + 1),  # half an ulp plus a bit in limb 0 only: the sticky word decides
        (top + 1, (1 << p) - 2),  # rounds up to 2^p: exponent carry
        (1000 << (p - 10), 999 << (p - 10)),  # small integers lifted: exact product
        (int("80" * (p // 8), 16), int("7f" * (p // 8), 16) | top),  # digits at the balanced range's ends
        (int("ff80" * (p // 16), 16), int("80ff" * (p // 16), 16)),
    ]
    return cases


@pytest.mark.parametrize("KD", KDS)
def test_operands_sums_limbs_and_rounding(KD):
    g = Geo(KD)
    p, NL = 8 * KD, g.NL
    exact_paths = lazy_paths = 0
    for z, b in operands(KD, 2000 + KD):
        A = a_row(z, g)
        e, cz = balanced(z, KD)
        assert cz == 1
        assert [A[KD - 1 - s] for s in range(KD)] == e  # digit s at K position KD - 1 - s
        assert sum(v << (8 * s) for s, v in enumerate(e)) + (1 << p) == z
        bt = b_tilde(b, g)
        eb, cb = balanced(b, KD)
        assert bt == eb + [cb] and cb == 1
        D, absum = mma_sums(A, hankel_buffer(bt, g), extra_buffer(b, g), g)
        # against the plain convolution z' * b~ plus the raw digits of b
        # (2^p b) and, in the upper tiles, the bias the MMA adds
        for r in range(2 * KD):
            c = sum(e[s] * bt[r - s] for s in range(KD) if 0 <= r - s <= KD)
            assert -4161536 <= c <= 4194304  # the digit convolution alone: at most 256 products
            raw = (b >> (8 * (r - KD))) & 255 if r >= KD else 0
            assert -4161536 <= c + raw <= 4194559
            bias = K_MAGIC if r // 128 >= g.XT0 else 0
            assert D[r] == c + raw + bias
            assert absum[r] <= 2 ** 22 + 128  # every partial sum of the digit steps is an exact fp32 integer
        assert sum(int(D[r] - (K_MAGIC if r // 128 >= g.XT0 else 0)) << (8 * r) for r in range(2 * KD)) == z * b
        up, l63, sticky, exact_path, acc = epilogue(fp32_words(D, g), g)
        P = z * b
        assert acc == 0  # the product fits its 2 NL limbs
        for q in range(NL):
            assert up[q] == (P >> (32 * (NL + q))) & MASK
        assert l63 == (P >> (32 * (NL - 1))) & MASK
        assert (sticky != 0) == (P & ((1 << (32 * (NL - 1))) - 1) != 0)
        exact_paths += exact_path
        lazy_paths += not exact_path
        assert round_product(up, l63, sticky, NL) == rne_product(z, b, p)
    assert lazy_paths >= 4 and exact_paths >= 2  # both epilogue paths ran


@pytest.mark.parametrize("KD", KDS)
def test_lazy_low_half_bound(KD):
    """The sums below chunk K0 (positions r < R = 32 K0 = KD - 32, each with at
    most r + 1 digit products in [-16256, 16384] and no raw digit of b) move
    limb NL - 8 by a carry in [-(2^14 - 1), 2^14 - 1]: so when bits [14, 224)
    of limbs NL - 8 .. NL - 2 hold a one and a zero, no carry or borrow leaves
    them and they stay non-zero (the sticky bit is 1)."""
    g = Geo(KD)
    R = 32 * g.K0
    assert R == KD - 32 and R <= KD
    pos = sum((r + 1) * 16384 * 256 ** r for r in range(R))
    neg = sum((r + 1) * 16256 * 256 ** r for r in range(R))
    assert pos < 2 ** 14 * 256 ** R
    assert neg <= (2 ** 14 - 1) * 256 ** R
    # the window argument: F mod 2^224 in [2^14, 2^224 - 2^14 - 1] plus a
    # carry in [-(2^14 - 1), 2^14 - 1] stays in [1, 2^224 - 2]
    lo, hi = 2 ** 14, 2 ** 224 - 2 ** 14 - 1
    assert lo - (2 ** 14 - 1) >= 1 and hi + 2 ** 14 - 1 <= 2 ** 224 - 2


@pytest.mark.parametrize("KD", KDS)
def test_tile_k_ranges_and_cores(KD):
    """Every non-zero term of tile t (positions [128 t, 128 t + 128), K
    position k' = KD - 1 - s meeting b~[r - s]) lies in the tile's K steps;
    merged tiles share their range; only cores KD/8 - 1 .. KD/4 - 1 meet b~'s
    digits (the others keep the set-up's zeros); the extra K step covers the
    positions >= KD; the MMA work per product."""
    g = Geo(KD)
    for t in range(g.TILES):
        lo, hi = g.ks_lo(t), g.ks_hi(t)
        assert 0 <= lo < hi <= KD // 16
        for r in range(128 * t, 128 * t + 128):
            for s in range(KD):
                if 0 <= r - s <= KD:
                    assert 16 * lo <= KD - 1 - s < 16 * hi
    for d in range(g.NCORE):
        meets = any(0 <= 8 * d + nn + kk - KD + 1 <= KD for nn in range(8) for kk in range(8))
        assert meets == (KD // 8 - 1 <= d <= KD // 4 - 1)
    assert 128 * g.XT0 <= KD
    macs = sum((g.ks_hi(t) - g.ks_lo(t)) * 16 * 128 * cnt for t, cnt in g.groups())
    macs += (g.TILES - g.XT0) * 16 * 128
    # the issued MMA work per product against the KD^2 digit products: the
    # Hankel corners skipped per 16-digit K step and 128-position tile, plus
    # the extra K step, cost most at the short mantissas
    assert macs / (KD * KD) == {64: 2.5, 128: 2.125, 256: 1.5625}[KD]


def test_carry_lookahead_formula():
    """carry_mask against a lane-by-lane carry chain on random generate and
    propagate patterns (disjoint, as the builders' ballots are)."""
    g = random.Random(7)
    for _ in range(2000):
        gen = g.getrandbits(32)
        prop = g.getrandbits(32) & ~gen
        if g.random() < 0.3:
            prop = (~gen) & MASK  # long propagate runs
        for inject in (0, 1):
            cm = carry_mask(gen, prop, inject)
            c = inject
            for l in range(32):
                assert (cm >> l) & 1 == c
                c = 1 if (gen >> l) & 1 or ((prop >> l) & 1 and c) else 0
            assert (cm >> 32) & 1 == c


@pytest.mark.parametrize("KD", KDS)
def test_a_operand_layout(KD):
    """A's rows as the epilogue warps write them (row r at (r >> 3) KA 16 +
    (r & 7) 16, K position k' at (k' >> 3) 128 + (k' & 7) 2) are what the
    descriptor reads (start 256 ks, leading offset 128, stride offset KA 16),
    and no two elements share a byte."""
    g = Geo(KD)
    KA = g.KA

    def row_addr(r, k):
        return (r >> 3) * (KA * 16) + (r & 7) * 16 + (k >> 3) * 128 + (k & 7) * 2

    seen = set()
    for r in range(128):
        for k in range(KA):
            a = row_addr(r, k)
            assert a not in seen
            seen.add(a)
    assert max(seen) < 128 * KA * 2
    for ks in range(KA // 16):
        for m in range(0, 128, 5):
            for kl in range(16):
                a = 256 * ks + (m // 8) * (KA * 16) + (kl // 8) * 128 + (m % 8) * 16 + (kl % 8) * 2
                assert a == row_addr(m, 16 * ks + kl)


@pytest.mark.parametrize("NL", [16, 32, 64])
def test_row_tile_swizzle(NL):
    """RowT: every row's 16-byte chunks land on distinct bytes of the 32-row
    tile, and for any chunk index eight consecutive rows (aligned) use eight
    different 16-byte bank quads, so one thread per row reads without bank
    conflicts."""
    TILE = 32 * NL * 4

    def off(r, kk):
        if NL >= 32:
            return (kk >> 3) * 4096 + r * 128 + (((kk & 7) ^ (r & 7)) << 4)
        return r * 64 + ((kk ^ ((r >> 1) & 3)) << 4)

    seen = set()
    for r in range(32):
        for kk in range(NL // 4):
            o = off(r, kk)
            assert o % 16 == 0 and 0 <= o < TILE and o not in seen
            seen.add(o)
    assert len(seen) * 16 == TILE
    for kk in range(NL // 4):
        for r0 in range(0, 32, 8):
            quads = {(off(r, kk) % 128) // 16 for r in range(r0, r0 + 8)}
            assert len(quads) == 8


def test_constants():
    """kOff, the magic constant and the per-limb constant kC from their
    definitions; the biased window [2^23, 2^24) holds every column sum."""
    assert K_OFF == 4177920
    assert np.float32(K_MAGIC) == K_MAGIC == 12566528
    assert K_C == 152833374535680
    assert -4161536 + K_MAGIC >= 2 ** 23 and 4194559 + K_MAGIC < 2 ** 24
    for v in range(-128, 257):  # every digit value is exact in bf16
        bf16_exact(v)


def simulate_tmem_handoff(KD, TB, nc, seed):
    """The MMA issuer and the epilogue of one block over nc columns with
    mbarrier parity waits, in a random interleaving: column c writes buffer
    c % TB (tile slots (c % TB) TILES + t); the issuer waits, from column TB
    on, for the empty barriers of its slots with parity (c / TB - 1) & 1 and
    commits a full barrier per tile group; the epilogue waits for the full
    barrier of tile T0 and then of each later tile with parity (c / TB) & 1,
    reads chunks K0 .. NCH - 1 (and, on the exact path, the chunks below K0),
    and releases each tile after its last chunk (the tiles up to T0 once the
    K0 chunk is done).  Checks that every read sees its own column's sums,
    that no tile is written while the previous column in it is unread, and
    that no barrier is ever two phases ahead of its waiter (a parity wait
    could not tell)."""
    g = Geo(KD)
    rnd = random.Random(seed)
    TILES, K0, NCH = g.TILES, g.K0, g.NCH
    T0 = K0 >> 2
    full = [0] * 4  # completions per slot
    empty = [0] * 4
    owner = [None] * 4  # column whose sums a slot holds
    released = [set() for _ in range(4)]  # columns whose sums a slot no longer needs

    def wait(bar, slot, j):
        """The j-th completion (parity j & 1) of a barrier: a wait point."""
        while True:
            done = bar[slot]
            assert done <= j + 1, "barrier two phases ahead of its waiter"
            if done == j + 1:
                return
            yield

    def issuer():
        for c in range(nc):
            tu = (c % TB) * TILES
            for t, cnt in g.groups():
                if c >= TB:
                    for q in range(cnt):
                        yield from wait(empty, tu + t + q, c // TB - 1)
                for q in range(cnt):
                    slot = tu + t + q
                    assert owner[slot] is None or owner[slot] in released[slot], "tile overwritten while unread"
                    owner[slot] = c
                yield
                for q in range(cnt):
                    full[tu + t + q] += 1

    def epilogue(exact_cols):
        for c in range(nc):
            tu = (c % TB) * TILES
            yield from wait(full, tu + T0, c // TB)
            for t in range(T0 + 1):
                assert owner[tu + t] == c  # committed in issue order: tiles up to T0 hold column c
            for k in range(K0, NCH):
                if k > K0 and (k & 3) == 0:
                    yield from wait(full, tu + (k >> 2), c // TB)
                assert owner[tu + (k >> 2)] == c
                if k == K0 and c in exact_cols:
                    for kk in range(K0):
                        assert owner[tu + (kk >> 2)] == c
                yield
                if k == K0:
                    for t in range(T0):
                        released[tu + t].add(c)
                        empty[tu + t] += 1
                    if (K0 & 3) == 3:
                        released[tu + T0].add(c)
                        empty[tu + T0] += 1
                elif (k & 3) == 3:
                    released[tu + (k >> 2)].add(c)
                    empty[tu + (k >> 2)] += 1

    agents = [issuer(), epilogue({c for c in range(nc) if rnd.random() < 0.3})]
    alive = [True, True]
    for _ in range(100000):  # a wait that never ends shows up as running out of steps
        if not any(alive):
            break
        i = rnd.choice([a for a in range(2) if alive[a]])
        try:
            next(agents[i])
        except StopIteration:
            alive[i] = False
    assert not any(alive), "the roles wait for each other"
    for s in range(TB * TILES):
        assert full[s] == empty[s] == len(range(s // TILES, nc, TB))  # every use completed and released


@pytest.mark.parametrize("KD", KDS)
def test_tensor_memory_buffers_and_barrier_parities(KD):
    """The kernel's buffering: two tensor-memory buffers at p = 512 and 1024
    (a column's tiles fill at most half of the 512 columns), one at p = 2048;
    the slot and parity arithmetic of both roles under random interleavings,
    and with one buffer forced at every precision."""
    g = Geo(KD)
    TB = 2 if g.TILES <= 2 else 1
    assert TB * g.TILES <= 4 and TB * g.TILES * 128 <= 512
    assert {64: 2, 128: 2, 256: 1}[KD] == TB
    for seed in range(40):
        simulate_tmem_handoff(KD, TB, 7, seed)
        simulate_tmem_handoff(KD, 1, 5, 100 + seed)
