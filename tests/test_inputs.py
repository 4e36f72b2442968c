"""Pins of the seeded input generator shared by the oracle, the tests and the
benchmark (CPU only).

  * mix64 is SplitMix64's output function: the sequential generator built on
    it (state += 0x9E3779B97F4A7C15, output mix64(state)) reproduces the
    published output sequences of the reference SplitMix64 for seeds 0 and
    1234567 (Steele, Lea and Flood, OOPSLA 2014; Vigna's public-domain
    splitmix64.c);
  * the stream is counter based: any window of counters equals the same slice
    of a longer draw;
  * uniforms carry 53 random bits in [0, 1);
  * Box--Muller normals have the standard normal's moments and one-sigma mass;
  * the "cos" start is m + amp cos(2 pi x) cos(2 pi y) [cos(2 pi z)] at the
    vertices, x fastest.
"""
import math

import numpy as np
import pytest

import ok_inputs as oi


def splitmix64(seed, count):
    with np.errstate(over="ignore"):
        return [int(oi.mix64(np.uint64(seed) + np.uint64(k + 1) * oi.GOLDEN)) for k in range(count)]


def test_mix64_reproduces_the_published_splitmix64_sequences():
    assert splitmix64(0, 4) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    assert splitmix64(1234567, 5) == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                                      4593380528125082431, 16408922859458223821]


def test_stream_is_counter_based():
    full = oi.bits(7, 1000)
    assert np.array_equal(oi.bits(7, 10, offset=500), full[500:510])
    assert np.array_equal(oi.uniform01(7, 3, offset=997), oi.uniform01(7, 1000)[997:])
    assert not np.array_equal(oi.bits(7, 100), oi.bits(8, 100))          # seeds give distinct streams
    assert len(np.unique(full)) == 1000


def test_uniforms_have_53_bits_in_the_unit_interval():
    u = oi.uniform01(3, 1 << 16)
    assert u.min() >= 0.0 and u.max() < 1.0
    scaled = u * 2.0 ** 53
    assert np.array_equal(scaled, np.floor(scaled))
    n = u.size
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 5 * math.sqrt(1 / 180 / n)              # Var of U^2-like terms: 1/180
    lo, hi = oi.uniform(3, 1000, -1.0, 1.0).min(), oi.uniform(3, 1000, -1.0, 1.0).max()
    assert -1.0 <= lo and hi < 1.0


def test_box_muller_normals_have_standard_moments():
    n = 1 << 20
    z = oi.normal(11, n)
    assert np.all(np.isfinite(z))
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2 / n)
    assert abs(np.mean(z ** 4) - 3.0) < 5 * math.sqrt(96 / n)             # Var(z^4) = 105 - 9
    p = math.erf(1 / math.sqrt(2))                                          # one-sigma mass 0.6827
    assert abs(np.mean(np.abs(z) < 1.0) - p) < 5 * math.sqrt(p * (1 - p) / n)


@pytest.mark.parametrize("dim", [2, 3])
def test_cos_start_closed_form(dim):
    n = 8
    wl = oi.Workload("cos_check", dim, n, 0.02, 100.0, 0.4, 0.5, 4e-4, 1, "cos", 0.02, 0, 30, 1e-8, 1e-10)
    u = oi.initial_u(wl)
    assert u.shape == ((n + 1) ** dim,)
    assert u[0] == pytest.approx(0.42)                                      # origin: all cosines 1
    k = n // 2                                                              # x = 1/2 at vertex index k
    assert u[k] == pytest.approx(0.38)                                      # cos(pi) = -1 in x only
    x = oi.nodal_coords(dim, n)
    assert np.allclose(x[1], [1.0 / n] + [0.0] * (dim - 1))                 # x fastest
    assert u == pytest.approx(0.4 + 0.02 * np.prod(np.cos(2 * np.pi * x), axis=1))
