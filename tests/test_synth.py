"""The seeded input generators: SplitMix64 against its published first outputs, the counter
mode's slicing, the Gaussian's moments, and the workload recipes (city batch, uneven
multi-box batch, bit order) that stand in for the paper's data."""
import numpy as np

import synth


def test_splitmix64_published_first_outputs():
    """SplitMix64 from state 0 (Steele, Lea and Flood's generator; the values every
    reference implementation prints) is mix64(k * GAMMA) for k = 1, 2, 3."""
    k = np.array([1, 2, 3], dtype=np.uint64)
    with np.errstate(over="ignore"):
        got = synth._mix64(k * synth.GAMMA)
    assert [int(v) for v in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_counter_mode_slices_regenerate():
    full = synth.splitmix64(5, 7, 1000)
    assert np.array_equal(synth.splitmix64(5, 7, 100, offset=450), full[450:550])
    assert not np.array_equal(synth.splitmix64(5, 8, 1000), full)      # streams differ
    assert not np.array_equal(synth.splitmix64(6, 7, 1000), full)      # seeds differ
    d = synth.lwe_draws(3, 50)
    tail = synth.lwe_draws(3, 20, offset=30)
    assert np.array_equal(d.mask[30:], tail.mask) and np.array_equal(d.noise[30:], tail.noise)


def test_uniform_bits_are_balanced():
    b = synth.bits(1, 2, 200000)
    assert abs(b.mean() - 0.5) < 0.005
    u = synth.uniform_u32(1, 3, 200000).astype(np.float64) / 2**32
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1 / 12) < 0.002


def test_gaussian_moments():
    sigma = 2.0 ** -15
    e = synth.gaussian_t32(2, 9, 200000, sigma).astype(np.int64)
    e = np.where(e >= 2**31, e - 2**32, e) / 2**32
    assert abs(e.mean()) < 5 * sigma / np.sqrt(len(e))
    assert abs(e.std() / sigma - 1) < 0.01
    assert not synth.gaussian_t32(2, 9, 10, 0.0).any()


def test_int_to_bits_is_lsb_first_twos_complement():
    assert synth.int_to_bits(6, 4).tolist() == [0, 1, 1, 0]
    assert synth.int_to_bits(-1, 5).tolist() == [1] * 5
    assert synth.int_to_bits(-2, 4).tolist() == [0, 1, 1, 1]


def test_city_batch_recipe():
    l, m = 16, 8
    qs = synth.city_batch(2, 400, l, m)
    inside = 0
    for k, q in enumerate(qs):
        x1, x2, y1, y2 = q.box
        assert 0 <= x1 < x2 < 2**l and 0 <= y1 < y2 < 2**l
        assert q.service.shape == (m,) and set(np.unique(q.service)) <= {0, 1}
        ins = x1 <= q.x < x2 and y1 <= q.y < y2
        assert ins == (k % 2 == 0), k            # even queries inside, odd ones outside
        inside += ins
        # outside points stay within the box widened by its own width on each side
        assert max(0, x1 - (x2 - x1)) <= q.x < min(2**l, x2 + (x2 - x1)) or ins
    assert inside == 200


def test_multibox_batch_recipe():
    qs = synth.multibox_batch(4, 300, m=16, max_boxes=128, widths=(16, 24, 32))
    ls = {q.l for q in qs}
    assert ls == {16, 24, 32}
    nbs = [len(q.boxes) for q in qs]
    assert min(nbs) >= 1 and max(nbs) <= 128 and np.mean(nbs) > 40      # ~U{1..128}, mean 64.5
    for q in qs:
        L = 1 << q.l
        assert 0 <= q.x < L and 0 <= q.y < L
        assert np.asarray(q.services).shape == (len(q.boxes), 16)
        for x1, x2, y1, y2 in q.boxes:
            assert 0 <= x1 <= x2 < L and 0 <= y1 <= y2 < L
