"""Host checks of the bit and float arithmetic the proximity kernels use.

* Byte-packed per-slot counters (count pass): a lane adds 1 << 8 (s % 4) to word
  s // 4 for every child slot s its record passes, over at most kTW tiles, and
  the warp adds its lanes' words (one reduction per word).  Checked: the sums
  decode to the per-slot counts, so no byte carries into the next.
* 16-bit record fields (biased by 2^15): a field becomes a float by placing its
  16 bits under the exponent of 1.5 * 2^23 (a byte permute with 0x4B40) and
  subtracting 1.5 * 2^23 + 2^15.  Checked exactly for all 65536 values.
* Rounding by a magic constant (emit pass): y + (1.5 * 2^23 + 2^15) in FP32 holds
  round-half-even(y) + 2^15 in its low 16 bits (|y| < 2^15), and the fused
  q * 0.5 + that constant holds the re-snap round-half-even(q / 2) + 2^15; the
  32-bit form y + 1.5 * 2^23 holds round-half-even(y) in its bits minus 0x4B400000.
  Checked on ties and random values, against Python's round (half to even).
* Child ranges (emit pass): one thread per child slot walks a block's tiles in
  order, takes one range per (cell, child) run with an atomic on the child's
  cursor and hands every tile its offset; positions of all blocks together are a
  permutation of [0, count) for every (cell, child).  Checked on random tile
  sequences.
"""
import numpy as np

KTW = 4          # tiles per warp (gv_tile.cuh)
KWARPS = 8


def f32(x):
    return np.float32(x)


def bits(x):
    return int(np.asarray(np.float32(x)).view(np.uint32))


def from_bits(b):
    return float(np.asarray(np.uint32(b)).view(np.float32))


def byte_perm(x, y, sel):
    src = [(x >> (8 * i)) & 255 for i in range(4)] + [(y >> (8 * i)) & 255 for i in range(4)]
    return sum(src[(sel >> (4 * i)) & 7] << (8 * i) for i in range(4))


MAGIC = 12582912.0
MAGIC16 = 12615680.0


def test_packed_counters_do_not_carry():
    rng = np.random.default_rng(0)
    for trial in range(200):
        p = 1.0 if trial == 0 else rng.random()
        passes = rng.random((32, KTW, 8)) < p            # lane, tile, slot
        words = [0, 0]
        for lane in range(32):
            w = [0, 0]
            for k in range(KTW):
                for s in range(8):
                    if passes[lane, k, s]:
                        w[s >> 2] += 1 << (8 * (s & 3))
            words[0] += w[0]
            words[1] += w[1]
        assert all(x < 2 ** 32 for x in words)
        counts = passes.sum(axis=(0, 1))
        for s in range(8):
            assert (words[s >> 2] >> (8 * (s & 3))) & 255 == counts[s]
    assert 32 * KTW < 256


def test_16bit_fields_to_float_exact():
    for q in range(-32768, 32768):
        u = q + 32768
        word = (u << 16) | 0x1234 if q % 2 else (0xABCD << 16) | u
        sel = 0x5432 if q % 2 else 0x5410
        b = byte_perm(word, 0x4B40, sel)
        v = f32(f32(from_bits(b)) - f32(MAGIC16))
        assert float(v) == q


def round_half_even(x):
    return int(round(x))           # Python rounds halves to even


def test_magic_rounding_and_resnap():
    rng = np.random.default_rng(1)
    ys = np.concatenate([np.arange(-40, 41) * 0.5, rng.uniform(-32000, 32000, 20000),
                         [32766.5, -32767.5, 0.4999999, -0.5000001]])
    for y in ys:
        y = float(f32(y))
        t = f32(f32(y) + f32(MAGIC16))                  # FP32 add, one rounding
        q = round_half_even(y)
        assert bits(t) & 0xFFFF == (q + 32768) & 0xFFFF, y
        assert float(f32(t - f32(MAGIC16))) == q
        if abs(y) < 2 ** 22:
            t32 = f32(f32(y) + f32(MAGIC))
            d = (bits(t32) - 0x4B400000) & 0xFFFFFFFF
            assert (d - (1 << 32) if d >= 1 << 31 else d) == q
    # the re-snap of an essential parameter when its step doubles: fma(q, 0.5, MAGIC16)
    for q in list(range(-300, 301)) + list(rng.integers(-32768, 32768, 5000)):
        q = int(q)
        exact = q * 0.5 + MAGIC16                        # exact in FP64, one FP32 rounding as in fma
        t = f32(exact)
        k = q >> 1
        want = k + ((q & 1) & (k & 1))                  # the integer re-snap of the 32-bit path
        assert want == round_half_even(q / 2)
        assert bits(t) & 0xFFFF == (want + 32768) & 0xFFFF


def walk_offsets(tile_cells, ballots, cursor, ns):
    """Python restatement of the emit pass's phase 2 for one block."""
    nt = len(tile_cells)
    off = np.zeros((nt, ns), np.int64)
    for s in range(ns):
        cur, start, run = -1, 0, 0
        for i in range(nt + 1):
            cl = tile_cells[i] if i < nt else -2
            if cl != cur:
                if cur >= 0 and run:
                    base = cursor[cur, s]
                    cursor[cur, s] += run
                    off[start:i, s] += base
                cur, run, start = cl, 0, i
            if i < nt:
                off[i, s] = run
                run += bin(ballots[i][s]).count("1")
    return off


def test_child_ranges_are_permutations():
    rng = np.random.default_rng(2)
    ns = 8
    for trial in range(60):
        ncell = int(rng.integers(1, 7))
        sizes = rng.integers(1, 200, ncell)
        tile_cells, tile_valid = [], []
        for cl, n in enumerate(sizes):
            for t in range((n + 31) // 32):
                tile_cells.append(cl)
                tile_valid.append(min(32, n - 32 * t))
        ballots = []
        for v in tile_valid:
            m = (1 << v) - 1
            ballots.append([int(rng.integers(0, 2 ** 32)) & m for _ in range(ns)])
        cursor = np.zeros((ncell, ns), np.int64)
        nb = 4 * KWARPS * KTW // 8                      # blocks of various sizes over the same tiles
        positions = {}
        for b0 in range(0, len(tile_cells), nb):
            tc = tile_cells[b0:b0 + nb]
            bl = ballots[b0:b0 + nb]
            off = walk_offsets(tc, bl, cursor, ns)
            for i, cl in enumerate(tc):
                for s in range(ns):
                    b = bl[i][s]
                    for lane in range(32):
                        if (b >> lane) & 1:
                            pos = off[i, s] + bin(b & ((1 << lane) - 1)).count("1")
                            positions.setdefault((cl, s), []).append(pos)
        for (cl, s), ps in positions.items():
            assert sorted(ps) == list(range(len(ps)))
            assert cursor[cl, s] == len(ps)
