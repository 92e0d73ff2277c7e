"""The learned-CDF path: hand-written forward/backward against the double-precision reference,
training that lowers the loss, bit-exact sorts (the model only changes bucket balance), and
what the trained model gains over its untrained starting point."""

import numpy as np
import pytest
import torch

import oracle
import paper_2106_05123_gb300 as pdq
import workloads
from gpu_helpers import bits
from oracle import learned as L

pytestmark = pytest.mark.gpu


def _sorted_sample(n, seed):
    x, _ = workloads.mixture_f32(n, seed)
    x = np.sort(x)
    mu = float(x[x.size // 2])
    sigma = float(np.float32(x[-1]) - np.float32(x[0]))
    return x, np.float32(mu), np.float32(sigma)


def _normalised_f32(x, mu, sigma):
    """The normalised keys exactly as the float32 kernels form them: fl(fl(x - mu) / sigma)."""
    return (x.astype(np.float32) - np.float32(mu)) / np.float32(sigma)


def _grad_case(x, mu, sigma, seed, noise):
    """GPU loss and gradient, and the float64 reference evaluated at the same float32-rounded
    normalised keys (mu = 0, sigma = 1 on the already normalised points)."""
    rng = np.random.default_rng(seed)
    theta = (L.init_theta(x.astype(np.float64), float(mu), float(sigma)) + rng.normal(0, noise, 48))
    theta = theta.astype(np.float32)
    t = ((np.arange(x.size) + 0.5) / x.size).astype(np.float32)
    loss_gpu, g_gpu = pdq.pdq_learned_loss_grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(),
                                                theta, float(mu), float(sigma))
    xn = _normalised_f32(x, mu, sigma).astype(np.float64)
    loss_ref, g_ref = L.loss_grad(theta.astype(np.float64), xn, t.astype(np.float64), 0.0, 1.0)
    return loss_gpu, np.array(g_gpu), loss_ref, g_ref


@pytest.mark.parametrize("seed", range(3))
def test_gradient_parity_with_reference(seed):
    """Well-conditioned data (N(0,1) keys, ramps of width ~1/16 of the range): the float32
    forward/backward matches the float64 reference to 1e-4 relative."""
    x = np.sort(workloads.normal_f32_specials(8192, 30 + seed, frac=0.0)[0])
    mu, sigma = np.float32(x[x.size // 2]), np.float32(x[-1] - x[0])
    loss_gpu, g_gpu, loss_ref, g_ref = _grad_case(x, mu, sigma, seed, 0.1)
    assert abs(loss_gpu - loss_ref) <= 1e-4 * max(1e-3, abs(loss_ref))
    assert np.linalg.norm(g_gpu - g_ref) <= 1e-4 * max(1e-3, np.linalg.norm(g_ref))


@pytest.mark.parametrize("seed", range(4))
def test_gradient_parity_on_mixture(seed):
    """On the mixture some ramps are very steep (clusters of width 1e-2 in a range of ~1e4), so
    the float32 rounding of a normalised key moves it by a visible fraction of such a ramp.  The
    reference therefore takes the same rounded normalised keys the kernels form; everything after
    that rounding must agree with the float64 reference to 1e-4 relative."""
    x, mu, sigma = _sorted_sample(8192, 10 + seed)
    loss_gpu, g_gpu, loss_ref, g_ref = _grad_case(x, mu, sigma, seed, 0.1)
    assert abs(loss_gpu - loss_ref) <= 1e-4 * max(1e-3, abs(loss_ref))
    assert np.linalg.norm(g_gpu - g_ref) <= 1e-4 * max(1e-3, np.linalg.norm(g_ref))


def test_training_lowers_the_loss_and_folds_consistently():
    x, _, _ = _sorted_sample(1 << 18, 5)
    out = pdq.pdq_learned_train(torch.from_numpy(x).cuda(), steps=64, batch=16384)
    assert out["loss_last"] < out["loss_first"]
    mu, sigma = out["mu"], out["sigma"]
    t = (np.arange(x.size) + 0.5) / x.size
    th0 = L.init_theta(x.astype(np.float64), mu, sigma)
    th1 = np.array(out["theta"], dtype=np.float64)
    mse0 = L.loss(th0, x, t, mu, sigma) / x.size
    mse1 = L.loss(th1, x, t, mu, sigma) / x.size
    assert mse1 < mse0
    # folded inference weights: a = softmax(alpha), w' = exp(omega) / sigma, t = mu + sigma c
    alpha, omega, c = L.split(th1)
    assert np.allclose(out["a"], L.softmax(alpha), rtol=1e-4, atol=1e-6)
    assert np.allclose(out["w"], np.exp(omega) / sigma, rtol=1e-4)
    assert np.allclose(out["t"], mu + sigma * c, rtol=1e-5, atol=1e-3)


def _learned_sort(keys):
    dk = torch.from_numpy(keys.copy()).cuda()
    st = pdq.pdq_sort_keys_learned(dk)
    torch.cuda.synchronize()
    return dk.cpu().numpy(), st


@pytest.mark.parametrize("n", [16385, 1 << 20, 3_000_001])
def test_learned_sort_is_exact_on_mixture(n):
    keys, _ = workloads.mixture_f32(n, 7)
    got, st = _learned_sort(keys)
    want = keys.copy()
    oracle.pdqsort(want)
    assert np.array_equal(bits(got), bits(want))
    assert st["learned_overflow"] >= 0


@pytest.mark.parametrize("kind", ["specials", "normal", "three_values", "uniform_bits", "sorted"])
def test_learned_sort_is_exact_on_hard_inputs(kind):
    n = 1 << 20
    if kind == "specials":
        keys, _ = workloads.normal_f32_specials(n, 3, frac=0.01)
    elif kind == "normal":
        keys, _ = workloads.normal_f32_specials(n, 4, frac=0.0)
    elif kind == "three_values":  # every key in very few buckets: the repair does all the work
        keys = np.array([-1.5, 0.25, 1e30], dtype=np.float32)[workloads.splitmix64(5, n) % np.uint64(3)]
    elif kind == "uniform_bits":  # all float bit patterns, NaNs included
        keys = workloads.uniform_bits(n, np.uint32, 6).view(np.float32)
    else:
        keys = np.sort(workloads.mixture_f32(n, 8)[0])
    got, st = _learned_sort(keys)
    want = keys.copy()
    oracle.pdqsort(want)
    assert np.array_equal(bits(got), bits(want))


def test_trained_model_gains_over_its_starting_point():
    """What training buys over the untrained network (ramps on the sixteenths of the sample), on
    fresh keys of the same mixture: a lower squared error to the empirical CDF, and the share of
    keys that land in buckets needing the exact repair (more than 4x the mean load)."""
    x, _, _ = _sorted_sample(1 << 18, 11)
    out = pdq.pdq_learned_train(torch.from_numpy(x).cuda(), steps=64, batch=16384)
    mu, sigma = out["mu"], out["sigma"]
    big = np.sort(workloads.mixture_f32(1 << 20, 11)[0]).astype(np.float64)  # same mixture
    t = (np.arange(big.size) + 0.5) / big.size
    th0 = L.init_theta(x.astype(np.float64), mu, sigma)
    th1 = np.array(out["theta"], dtype=np.float64)

    def overflow_fraction(theta):
        counts = np.bincount(L.buckets(theta, big, mu, sigma), minlength=4096)
        return counts[counts > 4 * big.size / 4096].sum() / big.size

    mse0, mse1 = L.loss(th0, big, t, mu, sigma) / big.size, L.loss(th1, big, t, mu, sigma) / big.size
    f0, f1 = overflow_fraction(th0), overflow_fraction(th1)
    print(f"CDF mse: untrained {mse0:.3e}, trained {mse1:.3e}; "
          f"keys in overflowing buckets: untrained {f0:.4f}, trained {f1:.4f}")
    assert mse1 < mse0
