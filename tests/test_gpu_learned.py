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


def _total_order_codes(x: np.ndarray) -> np.ndarray:
    """float32 keys as unsigned integers in IEEE totalOrder (test-side helper)."""
    b = x.view(np.uint32).astype(np.uint64)
    neg = (b >> np.uint64(31)) == 1
    return np.where(neg, np.uint64(0xFFFFFFFF) - b, b | np.uint64(0x80000000))


def test_trained_model_gain_at_equal_sample_budget():
    """What the trained network buys, on keys of the mixture workload, from one 1% sample:
    bucket balance (max / mean keys of the 4096 buckets) and CDF error of the trained model
    against its untrained starting point, with the sampled-splitter method at the same sample
    budget (4095 sample quantiles) and the device times of both sorts reported beside them.
    Training must improve on its starting point; the comparison with sampled splitters is
    measured and printed alongside: the test asserts the CDF gain, the other figures are
    recorded (on this mixture the splitters balance better and the plain path is faster)."""
    n, nb = 1 << 22, 4096
    keys, _ = workloads.mixture_f32(n, 13)
    m = n // 100
    pos = (workloads.splitmix64(workloads.substream(13, 7), m) % np.uint64(n)).astype(np.int64)
    sample = keys[pos].copy()
    oracle.pdqsort(sample)
    out = pdq.pdq_learned_train(torch.from_numpy(sample).cuda(), steps=24, batch=32768)
    mu, sigma = out["mu"], out["sigma"]
    fin = sample[np.isfinite(sample)].astype(np.float64)
    th0 = L.init_theta(fin, mu, sigma)
    th1 = np.array(out["theta"], dtype=np.float64)

    def balance(counts):
        return counts.max() / (n / nb)

    b0 = np.bincount(L.buckets(th0, keys, mu, sigma, nb), minlength=nb)
    b1 = np.bincount(L.buckets(th1, keys, mu, sigma, nb), minlength=nb)
    codes = _total_order_codes(keys)
    spl = _total_order_codes(sample)[((np.arange(1, nb) * m) // nb)]
    bs = np.bincount(np.searchsorted(spl, codes, side="right"), minlength=nb)
    srt = np.sort(keys[np.isfinite(keys)]).astype(np.float64)
    t = (np.arange(srt.size) + 0.5) / srt.size
    mse0 = L.loss(th0, srt, t, mu, sigma) / srt.size
    mse1 = L.loss(th1, srt, t, mu, sigma) / srt.size

    def device_ms(fn):
        d = torch.from_numpy(keys).cuda()
        ts = []
        for _ in range(4):
            d.copy_(torch.from_numpy(keys))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn(d)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts[1:]))

    t_learned = device_ms(lambda d: pdq.pdq_sort_keys_learned(d))
    t_plain = device_ms(lambda d: pdq.pdq_sort_keys(d))
    print(f"max/mean bucket: untrained {balance(b0):.2f}, trained {balance(b1):.2f}, "
          f"sampled splitters {balance(bs):.2f}; CDF mse untrained {mse0:.3e}, trained {mse1:.3e}; "
          f"device ms learned {t_learned:.3f}, plain {t_plain:.3f}")
    assert mse1 < mse0
