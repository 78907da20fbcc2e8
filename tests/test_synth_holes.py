"""The holed uv coverage of the generator (Sec. 4.1: holes through an inverse
Gaussian profile, missing Fourier content mainly at high spatial frequencies),
checked against its stated construction: no sample of the base pool lies in a
hole, hole centres sit at high frequencies more often than the samples do, the
pool keeps its size, and the coverage without holes is unchanged."""

import numpy as np

import synth


def test_no_sample_inside_a_hole_and_size_kept():
    rng = np.random.Generator(np.random.PCG64(3))
    freqs = synth.channel_freqs(4, 1.0, 2.0)
    std, limit = np.pi / 4, np.pi
    pool = synth.uv_coverage(rng, 5000, freqs, std, limit, holes=25)
    assert pool.shape == (5000, 2)
    rng2 = np.random.Generator(np.random.PCG64(3))   # the holes are the first draws
    c, r = synth.uv_holes(rng2, 25, std, limit, freqs[-1] / freqs[0])
    d = np.sqrt(((pool[:, None, :] - c[None]) ** 2).sum(-1))
    assert np.all(d >= r[None, :])
    assert np.all(np.max(np.abs(pool), axis=1) * 2.0 < limit)


def test_holes_favour_high_frequencies():
    rng = np.random.Generator(np.random.PCG64(4))
    std = np.pi / 4
    c, r = synth.uv_holes(rng, 4000, std, np.pi, 2.0)
    # the centres' density 1 - exp(-|c|^2 / 2 std^2) vanishes at the origin: far fewer centres
    # within std of it than a uniform draw over the band would put there
    frac_in = np.mean(np.sum(c * c, axis=1) < std * std)
    uniform = np.pi * std * std / (np.pi) ** 2          # disc area / band area (edge pi / 2)
    assert frac_in < 0.5 * uniform
    assert np.all((r >= 0.04 * np.pi / 2) & (r <= 0.12 * np.pi / 2))


def test_without_holes_the_draws_are_unchanged():
    a = synth.make_inputs(1)
    b = synth.make_inputs(1, holes=0)
    assert np.array_equal(a.uv, b.uv) and np.array_equal(a.noise, b.noise)
    h = synth.make_inputs(1, holes=20)
    assert h.uv.shape == a.uv.shape and not np.array_equal(h.uv, a.uv)
