"""The segmented sort (key descending, then id ascending) against numpy's
lexicographic sort, at the lengths where its strategy changes: the warp and
tile classes, long segments split into sample-sort buckets, segments so long
that their buckets are split again, and the tie patterns that decide bucket
boundaries by id alone."""
import numpy as np
import pytest

import paper_2012_11188_gb300 as gs

pytestmark = pytest.mark.gpu


def lexsorted(keys, ids, off):
    want_k, want_i = keys.copy(), ids.copy()
    for a, b in zip(off[:-1], off[1:]):
        if b - a > 1:
            o = np.lexsort((want_i[a:b], -want_k[a:b]))
            want_k[a:b], want_i[a:b] = want_k[a:b][o], want_i[a:b][o]
    return want_k, want_i


def device_sorted(keys, ids, off):
    import torch
    k = torch.from_numpy(keys).cuda()
    v = torch.from_numpy(ids).cuda()
    gs.sort_segments_desc(k, v, torch.from_numpy(off).cuda())
    return k.cpu().numpy(), v.cpu().numpy()


def check(keys, ids, lens):
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    got_k, got_i = device_sorted(keys, ids, off)
    want_k, want_i = lexsorted(keys, ids, off)
    assert np.array_equal(got_k, want_k)
    assert np.array_equal(got_i, want_i)


def test_lengths_around_every_class_and_bucket_boundary():
    rng = np.random.default_rng(11)
    lens = np.array([0, 1, 2, 31, 32, 33, 255, 256, 257, 1023, 1024, 1025, 4095, 4096, 4097,
                     8191, 8192, 8193, 16385, 100_000, 3_000_000, 7, 4097])
    total = int(lens.sum())
    keys = rng.random(total)
    ids = rng.permutation(total).astype(np.int32)
    check(keys, ids, lens)


@pytest.mark.parametrize("pattern", ["equal", "two_values", "ascending", "descending",
                                     "rounded"])
def test_tie_patterns_in_long_segments(pattern):
    rng = np.random.default_rng(12)
    lens = np.array([50_000, 4097, 300_000, 12])
    total = int(lens.sum())
    if pattern == "equal":  # every bucket boundary is decided by the id
        keys = np.full(total, 0.5)
    elif pattern == "two_values":
        keys = rng.choice([0.25, 0.75], total)
    elif pattern == "ascending":
        keys = np.sort(rng.random(total))
    elif pattern == "descending":
        keys = np.sort(rng.random(total))[::-1].copy()
    else:
        keys = np.round(rng.random(total), 3)
    ids = rng.permutation(total).astype(np.int32)
    check(keys, ids, lens)


def test_ids_in_order_within_equal_keys():
    # already sorted input: the samples see a sorted segment
    n = 200_000
    keys = np.repeat(np.linspace(1.0, 0.0, 50), n // 50)
    ids = np.arange(n, dtype=np.int32)
    check(keys, ids, np.array([n]))


def test_segment_whose_buckets_are_split_again():
    # more than 8192 buckets of the expected length: the buckets average above
    # 4096 elements and most are split again one level down
    rng = np.random.default_rng(13)
    lens = np.array([36_000_000, 5000])
    total = int(lens.sum())
    keys = rng.random(total)
    ids = rng.permutation(total).astype(np.int32)
    check(keys, ids, lens)


def test_offsets_outside_the_arrays_are_refused_before_any_access():
    import torch
    keys = torch.rand(1000, dtype=torch.float64, device="cuda")
    ids = torch.arange(1000, dtype=torch.int32, device="cuda")
    before_k, before_i = keys.clone(), ids.clone()
    for off in ([0, 600, 1200], [0, 700, 500, 1000], [-4, 500, 1000]):
        o = torch.tensor(off, dtype=torch.int64, device="cuda")
        with pytest.raises(gs.ScanError):
            gs.sort_segments_desc(keys, ids, o, max_len=1200)
    assert torch.equal(keys, before_k) and torch.equal(ids, before_i)
