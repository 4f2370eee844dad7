"""Pins of the FP64 loss oracle (Eq. "rnd_loss"): SSIM identities, a
brute-force windowed SSIM, a closed form on constant images, the L1 terms,
and central finite differences of the whole loss."""
import numpy as np
import torch

from oracle import loss as OL


def test_gaussian_window_is_normalised_and_symmetric():
    g = OL.gaussian_1d().numpy()
    assert abs(g.sum() - 1) < 1e-15 and np.allclose(g, g[::-1], rtol=0, atol=1e-17)
    assert g.argmax() == 5 and len(g) == 11


def test_ssim_of_identical_images_is_one():
    rng = np.random.default_rng(0)
    x = torch.tensor(rng.uniform(0, 1, (3, 17, 23)))
    np.testing.assert_allclose(OL.ssim_map(x, x).numpy(), 1.0, atol=1e-12)


def test_ssim_matches_brute_force_window_sums():
    rng = np.random.default_rng(1)
    x, y = rng.uniform(0, 1, (9, 13)), rng.uniform(0, 1, (9, 13))
    ref = OL.ssim_brute(x, y)
    got = OL.ssim_map(torch.tensor(x[None]), torch.tensor(y[None])).numpy()[0]
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


def test_ssim_of_constant_images_interior_closed_form():
    a, b = 0.3, 0.7
    x = torch.full((1, 30, 30), a, dtype=torch.float64)
    y = torch.full((1, 30, 30), b, dtype=torch.float64)
    s = OL.ssim_map(x, y).numpy()[0]
    # away from the zero-padded border the variances vanish: S = (2ab + C1)/(a^2 + b^2 + C1)
    np.testing.assert_allclose(s[5:-5, 5:-5], (2 * a * b + OL.C1) / (a * a + b * b + OL.C1), rtol=1e-12)


def test_loss_terms_and_weights():
    rng = np.random.default_rng(2)
    c, t = rng.uniform(0, 1, (3, 12, 14)), rng.uniform(0, 1, (3, 12, 14))
    d, td = rng.uniform(1, 3, (12, 14)), rng.uniform(1, 3, (12, 14))
    lam1, lam2 = 0.9, 0.2
    L, _, _ = OL.window_loss_and_grads([c], [t], [d], [td], lam1, lam2)
    s = OL.ssim_brute(c[0], t[0]).mean() + OL.ssim_brute(c[1], t[1]).mean() + OL.ssim_brute(c[2], t[2]).mean()
    expect = lam1 * ((1 - lam2) * np.abs(c - t).mean() + lam2 * (1 - s / 3)) + (1 - lam1) * np.abs(d - td).mean()
    assert abs(L - expect) < 1e-12


def test_loss_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    c, t = rng.uniform(0, 1, (3, 8, 9)), rng.uniform(0, 1, (3, 8, 9))
    d, td = rng.uniform(1, 3, (8, 9)), rng.uniform(1, 3, (8, 9))
    # keep |c - t| and |d - td| away from the kinks of the absolute value
    c = np.where(np.abs(c - t) < 0.05, t + 0.1, c)
    d = np.where(np.abs(d - td) < 0.05, td + 0.1, d)
    _, gc, gd = OL.window_loss_and_grads([c], [t], [d], [td], 0.8, 0.2)
    h = 1e-6
    fc = np.zeros_like(c)
    for idx in np.ndindex(c.shape):
        cp, cm = c.copy(), c.copy()
        cp[idx] += h
        cm[idx] -= h
        fc[idx] = (OL.window_loss_and_grads([cp], [t], [d], [td], 0.8, 0.2)[0] -
                   OL.window_loss_and_grads([cm], [t], [d], [td], 0.8, 0.2)[0]) / (2 * h)
    assert np.linalg.norm(gc[0] - fc) / np.linalg.norm(fc) < 1e-7
    np.testing.assert_allclose(gd[0], 0.2 * np.sign(d - td) / d.size, rtol=1e-12)
