"""Pins of the oracle's per-step Gaussian noise (Alg. 2's z_i): the Box-Muller
map at points where it has a closed value, the distribution of the stream, the
counter layout, and the noisy tick against a random-walk closed form."""
import math

import numpy as np
from scipy import stats

from oracle import mpmi, philox, safety, sampling


def _words(v):
    """uint32 words whose top 24 bits are v (the low 8 bits are ignored)."""
    return (np.asarray(v, dtype=np.uint64) << np.uint64(8)).astype(np.uint32) | np.uint32(0x5A)


def test_box_muller_closed_values():
    # u1 = 1 (top bits 2^24 - 1): radius 0, whatever the angle
    n0, n1 = sampling.box_muller(_words([2 ** 24 - 1]), _words([12345]))
    assert n0[0] == 0.0 and n1[0] == 0.0
    # u1 = 2^-24 (top bits 0): radius sqrt(48 ln 2); u2 = 0 puts it all on the cosine
    r = math.sqrt(48.0 * math.log(2.0))
    n0, n1 = sampling.box_muller(_words([0]), _words([0]))
    assert n0[0] == r and n1[0] == 0.0
    # u2 = 1/4 and 1/2 rotate it onto the sine and the negative cosine
    n0, n1 = sampling.box_muller(_words([0, 0]), _words([2 ** 22, 2 ** 23]))
    assert abs(n0[0]) < 1e-15 and n1[0] == r
    assert n0[1] == -r and abs(n1[1]) < 1e-15
    # u1 = e^-1/2 is not a lattice value; u1 = 1/2 gives radius sqrt(2 ln 2)
    n0, _ = sampling.box_muller(_words([2 ** 23 - 1]), _words([0]))
    assert n0[0] == math.sqrt(2.0 * math.log(2.0))


def test_noise_is_standard_normal_and_independent():
    z = sampling.gaussian_noise(seed=7, stream=3, tick=11, n_slots=4096, H=12, n_noise=8)
    assert z.shape == (12, 4096, 8)
    flat = z.reshape(-1)
    assert abs(flat.mean()) < 0.01
    assert abs(flat.var() - 1.0) < 0.01
    assert stats.kstest(flat, "norm").pvalue > 1e-3
    # each coordinate, step and slot on its own is standard normal and uncorrelated
    for j in range(8):
        assert abs(z[..., j].std() - 1.0) < 0.03
    c = np.corrcoef(z.reshape(-1, 8).T)
    assert np.max(np.abs(c - np.eye(8))) < 0.02
    a, b = z[:-1].reshape(-1), z[1:].reshape(-1)       # consecutive steps
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.01
    # the radius of one pair is Rayleigh: r^2 = n0^2 + n1^2 is chi-square with 2 dof
    r2 = (z[..., 0] ** 2 + z[..., 1] ** 2).reshape(-1)
    assert stats.kstest(r2, "chi2", args=(2,)).pvalue > 1e-3


def test_noise_counter_layout_and_determinism():
    c = sampling.noise_counter(np.array([5]), tick=(3 << 32) + 9, step=7, block=1, stream=4)
    assert [int(w[0]) for w in c] == [5, 9, 3 + (7 << 16) + (1 << 25), 4]
    # the counters stay clear of every candidate counter (third word >= 2^16)
    assert int(sampling.noise_counter(np.array([0]), 2 ** 48 - 1, 1, 0, 0)[2][0]) >= 2 ** 16
    # block b of step t is the Box-Muller image of one Philox call
    w = philox.philox4x32(*sampling.noise_counter(np.arange(3), 21, 2, 0, 6), 99, 0)
    z = sampling.gaussian_noise(99, 6, 21, 3, 2, 4)
    n0, n1 = sampling.box_muller(w[0], w[1])
    n2, n3 = sampling.box_muller(w[2], w[3])
    assert np.array_equal(z[1], np.stack([n0, n1, n2, n3], axis=1))
    # deterministic, and every (seed, stream, tick) gives a different stream
    z2 = sampling.gaussian_noise(99, 6, 21, 3, 2, 4)
    assert np.array_equal(z, z2)
    for other in [(98, 6, 21), (99, 7, 21), (99, 6, 22)]:
        assert not np.allclose(sampling.gaussian_noise(*other, 3, 2, 4), z)
    # a shorter coordinate count is a prefix of the longer one
    assert np.array_equal(sampling.gaussian_noise(99, 6, 21, 3, 2, 3), z[..., :3])


def _drift(dt):
    return np.array([[1.0, dt], [0.0, 1.0]])   # z = (x, u): x' = x + dt u, u held


def test_zero_noise_is_the_noise_free_tick():
    rng = np.random.default_rng(2)
    samples = rng.uniform(-1, 1, (200, 1))
    spec = safety.SafetySpec(lo=np.array([-1.0]), hi=np.array([1.0]))
    a = mpmi.tick(_drift(0.05), "linear", [0.3], [0.7], samples, 40, spec, record=True)
    b = mpmi.tick(_drift(0.05), "linear", [0.3], [0.7], samples, 40, spec, record=True,
                  noise=np.zeros((40, 201, 1)))
    assert a.index == b.index and np.array_equal(a.ttv, b.ttv)
    assert np.array_equal(a.traj, b.traj, equal_nan=True)


def test_noisy_drift_is_a_random_walk():
    # x_t = x0 + t dt xi + sigma sum_{s<=t} n_s; the input coordinate is untouched,
    # and the noise of step t is in place before step t's safety test.
    dt, H, x0, sigma = 0.05, 30, 0.2, 0.04
    rng = np.random.default_rng(9)
    samples = rng.uniform(-1, 1, (150, 1))
    spec = safety.SafetySpec(lo=np.array([-1.0]), hi=np.array([1.0]))
    n = sampling.gaussian_noise(seed=5, stream=1, tick=3, n_slots=151, H=H, n_noise=1)
    r = mpmi.tick(_drift(dt), "linear", [x0], [0.1], samples, H, spec, record=True,
                  noise=sigma * n)
    cands = r.candidates[:, 0]
    steps = np.arange(1, H + 1)[:, None]
    walk = x0 + steps * dt * cands[None, :] + sigma * np.cumsum(n[:, :, 0], axis=0)
    inside = (walk > -1.0) & (walk < 1.0)
    want_ttv = np.where(inside.all(axis=0), H, np.argmin(inside, axis=0))
    assert np.array_equal(r.ttv, want_ttv)
    for i in range(151):
        t_end = min(r.ttv[i] + 1, H)
        assert np.allclose(r.traj[i, 1:t_end + 1, 0], walk[:t_end, i], rtol=0, atol=1e-12)
        assert np.all(r.traj[i, 1:t_end + 1, 1] == cands[i])
    # noise changes which candidates survive (the pin is not vacuous)
    free = mpmi.tick(_drift(dt), "linear", [x0], [0.1], samples, H, spec)
    assert not np.array_equal(free.ttv, r.ttv)
