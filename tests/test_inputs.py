"""The seeded input generator shared by both sides: Philox4x32-10 against its
published known-answer vectors, and the channel construction."""
import json
import os

import numpy as np

from paper_1505_04979_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    kat = json.load(open(os.path.join(GOLDEN, "philox_kat.json")))
    for v in kat["vectors"]:
        ctr = [int(c, 16) for c in v["ctr"]]
        key = [int(k, 16) for k in v["key"]]
        out = I.philox4x32_10([ctr[0]], [ctr[1]], [ctr[2]], [ctr[3]], key[0], key[1])
        assert [int(o[0]) for o in out] == [int(o, 16) for o in v["out"]]


def test_streams_and_codewords_are_independent():
    a = I.random_words(7, I.STREAM_INFO, np.arange(4), 8)
    b = I.random_words(7, I.STREAM_NOISE, np.arange(4), 8)
    c = I.random_words(7, I.STREAM_INFO, np.arange(2, 6), 8)
    assert not np.array_equal(a, b)
    assert np.array_equal(a[2:], c[:2])  # codeword k is the same wherever it is generated


def test_info_bits_respect_the_frozen_set():
    fz = np.zeros(64, np.uint8)
    fz[::3] = 1
    u = I.info_bits(3, np.arange(200), fz)
    assert np.all(u[:, fz == 1] == 0)
    assert 0.4 < u[:, fz == 0].mean() < 0.6


def test_gaussian_moments():
    z = I.gaussian(5, np.arange(400), 1000)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.01


def test_channel_llr():
    x = np.array([[0, 1, 0, 1]], np.uint8)
    z = np.zeros((1, 4))
    s = I.sigma(3.0, 0.5)
    llr = I.channel_llr(x, z, s)
    assert np.allclose(llr, [[2 / s**2, -2 / s**2, 2 / s**2, -2 / s**2]])
    assert llr.dtype == np.float32
