"""Host checks of the bit arithmetic the proximity kernels use inside a warp.

* Byte-packed per-slot counters (count pass): a record's slot mask is spread to one
  byte per slot with (x * 0x00204081) & 0x01010101 for four slots at a time, and the
  words of all records of a warp are added.  Checked: the spread is exact for every
  4-bit mask, and a warp's sums (32 lanes x 4 records) decode to the per-slot
  counts, so no byte carries into the next.
* Run masks (emit pass): a warp's lanes hold consecutive records and a cell's
  records are contiguous, so the lanes of one cell form a run; the kernel finds a
  lane's run from the ballot of run heads.  Checked against brute force on random
  sorted cell sequences with idle tail lanes.
"""
import numpy as np

FULL = 0xFFFFFFFF
RPT = 4          # records per thread in the count pass


def spread4(x):
    return (x * 0x00204081) & 0x01010101


def run_mask(keys, lane):
    """Python restatement of the kernel's run_mask for one lane (keys: per-lane
    cell, -1 for a lane without a record)."""
    heads = 0
    for i in range(32):
        prev = keys[i - 1] if i > 0 else keys[0]
        if i == 0 or prev != keys[i]:
            heads |= 1 << i
    upto = FULL if lane == 31 else ((2 << lane) - 1)
    start = (heads & upto).bit_length() - 1
    after = heads & ~upto & FULL
    if after:
        first_after = (after & -after).bit_length() - 1
        below_end = (1 << first_after) - 1
    else:
        below_end = FULL
    return below_end & ~((1 << start) - 1) & FULL


def test_spread4_exact():
    for x in range(16):
        want = sum(((x >> i) & 1) << (8 * i) for i in range(4))
        assert spread4(x) == want


def test_packed_warp_counts_do_not_carry():
    rng = np.random.default_rng(0)
    for trial in range(200):
        # worst cases included: every lane passes every slot for every record
        p = 1.0 if trial == 0 else rng.random()
        masks = (rng.random((32, RPT, 8)) < p)
        words = [0, 0]
        for lane in range(32):
            for k in range(RPT):
                m = sum(int(b) << s for s, b in enumerate(masks[lane, k]))
                words[0] += spread4(m & 15)
                words[1] += spread4((m >> 4) & 15)
        assert all(w < 2 ** 32 for w in words)
        counts = masks.sum(axis=(0, 1))
        for s in range(8):
            assert (words[s // 4] >> (8 * (s % 4))) & 255 == counts[s]
    assert 32 * RPT < 256


def test_run_mask_matches_brute_force():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        nrec = int(rng.integers(1, 33))
        ncells = int(rng.integers(1, 9))
        keys = sorted(int(x) for x in rng.integers(0, ncells, size=nrec)) + [-1] * (32 - nrec)
        for lane in range(32):
            want = 0
            # the maximal block of equal keys around this lane
            a = lane
            while a > 0 and keys[a - 1] == keys[lane]:
                a -= 1
            b = lane
            while b < 31 and keys[b + 1] == keys[lane]:
                b += 1
            for i in range(a, b + 1):
                want |= 1 << i
            assert run_mask(keys, lane) == want, (keys, lane)
