"""Bucket-domain refinement on the GPU: loss and gradients against the FP64 oracle, the
autograd Function against the C call, central differences of the GPU loss, and the
refinement loop reducing off-grid frequency error."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_1610_01050_gb300 as R
from paper_1610_01050_gb300.autograd import BucketResidual

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1610_01050_gb300 import build as B
    B.build()
    R.load_library()


def _setup(n, b, loops, true_f, true_a, noise, seed, df):
    rng = np.random.default_rng(seed)
    cube = O.tone_field(n, true_f, true_a)
    cube = cube + noise * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
    cube64 = cube.astype(np.complex64)
    f0 = (np.asarray(true_f) + df).astype(np.float32)
    a0 = (np.asarray(true_a) * (0.9 + 0.1j)).astype(np.complex64)
    plan = R.rsft_plan_create(R.make_desc(n, b, loops, seed=seed, atten_db=50.0, p_fa1=0.05, mu=1))
    x = torch.from_numpy(cube64).cuda()
    R.rsft_refine_prepare(plan, x)
    op = O.make_plan(n, b, loops, seed=seed, atten_db=50.0, pfa1=0.05, mu=1)
    return plan, x, cube64.astype(np.complex128), f0, a0, op


def _eval(plan, f0, a0):
    f = torch.from_numpy(f0).cuda()
    a = torch.from_numpy(a0).cuda()
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    gf = torch.zeros_like(f)
    ga = torch.zeros_like(a)
    hd = torch.zeros((len(a0), f0.shape[1] + 1), dtype=torch.float32, device="cuda")
    R.rsft_refine_eval(plan, f, a, loss=loss, grad_freq=gf, grad_amp=ga, hdiag=hd)
    torch.cuda.synchronize()
    return float(loss.item()), gf.cpu().numpy(), ga.cpu().numpy(), hd.cpu().numpy()


CASES = [
    ("2d", (32, 16), (8, 4), 3, [[0.2031, 0.4106], [0.6719, 0.0833]], [1.3 - 0.4j, 0.6 + 0.9j]),
    ("3d", (16, 16, 8), (4, 4, 2), 4, [[0.11, 0.52, 0.33], [0.71, 0.27, 0.81], [0.43, 0.91, 0.05]],
     [1.0 + 0.2j, -0.5 + 0.7j, 0.8 - 0.8j]),
    ("2d_wide", (128, 64), (16, 8), 5, [[0.301, 0.627], [0.702, 0.114]], [2.0 + 0.0j, 0.0 - 1.5j]),
]


@pytest.mark.parametrize("name,n,b,loops,tf,ta", CASES, ids=[c[0] for c in CASES])
def test_loss_and_gradient_match_the_oracle(name, n, b, loops, tf, ta):
    df = 0.6 / np.asarray(n, dtype=np.float64)  # 0.6 bin off in every dimension
    plan, _, cube, f0, a0, op = _setup(n, b, loops, np.asarray(tf), np.asarray(ta), 0.05, 3, df)
    loss, gf, ga, hd = _eval(plan, f0, a0)
    ref_loss = O.refine_loss(op, cube, f0.astype(np.float64), a0.astype(np.complex128))
    rgf, rgre, rgim = O.refine_grad(op, cube, f0.astype(np.float64), a0.astype(np.complex128))
    assert loss == pytest.approx(ref_loss, rel=1e-4)
    # every component within 1e-3 of the FP64 gradient (relative to itself; a floor of 1e-6 of the
    # largest component only for components that cancel to nearly zero)
    ramp = np.stack([rgre, rgim], axis=1)
    gamp = np.stack([ga.real, ga.imag], axis=1)
    scale = max(np.abs(rgf).max(), np.abs(ramp).max())
    for got, ref in ((gf, rgf), (gamp, ramp)):
        err = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-3 * scale)
        assert np.all(np.abs(got - ref) <= 1e-3 * np.abs(ref) + 1e-6 * scale), err.max()
    assert np.all(hd > 0)
    # the same GPU gradient against central differences of the FP64 oracle loss at h = 1e-4 (in bins for
    # the frequencies, absolute for the amplitudes), per component at 1e-3
    f64, a64 = f0.astype(np.float64), a0.astype(np.complex128)
    for k in range(len(a0)):
        for d in range(len(n)):
            h = 1e-4 / n[d]
            fp, fm = f64.copy(), f64.copy()
            fp[k, d] += h
            fm[k, d] -= h
            fd = (O.refine_loss(op, cube, fp, a64) - O.refine_loss(op, cube, fm, a64)) / (2 * h)
            assert abs(gf[k, d] - fd) <= 1e-3 * abs(fd) + 1e-6 * scale, (k, d, gf[k, d], fd)
        for unit, g in ((1.0, gamp[k, 0]), (1j, gamp[k, 1])):
            ap, am = a64.copy(), a64.copy()
            ap[k] += 1e-4 * unit
            am[k] -= 1e-4 * unit
            fd = (O.refine_loss(op, cube, f64, ap) - O.refine_loss(op, cube, f64, am)) / 2e-4
            assert abs(g - fd) <= 1e-3 * abs(fd) + 1e-6 * scale, (k, unit, g, fd)


def test_autograd_function_returns_the_library_gradient():
    n, b, loops, tf, ta = CASES[1][1:]
    plan, _, _, f0, a0, _ = _setup(n, b, loops, np.asarray(tf), np.asarray(ta), 0.05, 4, 0.02)
    loss, gf, ga, _ = _eval(plan, f0, a0)
    f = torch.from_numpy(f0).cuda().requires_grad_(True)
    ari = torch.view_as_real(torch.from_numpy(a0).cuda()).clone().requires_grad_(True)
    e = BucketResidual.apply(f, ari, plan)
    (g1, g2) = torch.autograd.grad(e, [f, ari])
    assert float(e.detach()) == pytest.approx(loss, rel=1e-6)
    np.testing.assert_array_equal(g1.cpu().numpy(), gf)
    np.testing.assert_array_equal(g2.cpu().numpy(), np.stack([ga.real, ga.imag], axis=1))


def test_gpu_loss_central_differences():
    """An extra check on the FP32 loss itself: its central differences (h = 0.01 bin) track the GPU
    gradient to 1e-2.  FP32 limits this one: the loss is a sum of squares near its minimum, so a
    difference of two FP32 losses at h = 1e-4 would be rounding; the 1e-3 agreement at h = 1e-4 is
    checked against the FP64 oracle's loss in test_loss_and_gradient_match_the_oracle."""
    n, b, loops, tf, ta = CASES[2][1:]
    plan, _, _, f0, a0, _ = _setup(n, b, loops, np.asarray(tf), np.asarray(ta), 0.05, 5, 0.3 / np.asarray(n))
    _, gf, ga, _ = _eval(plan, f0, a0)
    for k in range(len(a0)):
        for d in range(2):
            h = 0.01 / n[d]  # a hundredth of a bin
            fp, fm = f0.copy(), f0.copy()
            fp[k, d] += h
            fm[k, d] -= h
            fd = (_eval(plan, fp, a0)[0] - _eval(plan, fm, a0)[0]) / (2 * h)
            assert fd == pytest.approx(gf[k, d], rel=1e-2, abs=1e-3 * np.abs(gf).max())
        h = 1e-3 * abs(a0[k])
        for unit, g in ((1.0, ga[k].real), (1j, ga[k].imag)):
            ap, am = a0.copy(), a0.copy()
            ap[k] += h * unit
            am[k] -= h * unit
            fd = (_eval(plan, f0, ap)[0] - _eval(plan, f0, am)[0]) / (2 * h)
            assert fd == pytest.approx(g, rel=1e-2, abs=1e-3 * np.abs(ga).max())


def test_refinement_reduces_off_grid_frequency_error():
    n, b, loops = (256, 256), (16, 16), 8
    rng = np.random.default_rng(21)
    k = 6
    bins = np.stack([rng.choice(np.arange(8, 248, 40), k, replace=False),
                     rng.choice(np.arange(8, 248, 40), k, replace=False)], axis=1).astype(np.float64)
    true_f = (bins + rng.uniform(-0.45, 0.45, (k, 2))) / np.asarray(n)
    true_a = (rng.uniform(1.0, 2.0, k) * np.exp(2j * np.pi * rng.uniform(0, 1, k)))
    cube = O.tone_field(n, true_f, true_a) + 0.02 * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
    plan = R.rsft_plan_create(R.make_desc(n, b, loops, seed=21, atten_db=60.0, p_fa1=0.05, mu=1))
    x = torch.from_numpy(cube.astype(np.complex64)).cuda()
    f = torch.from_numpy((np.round(true_f * np.asarray(n)) / np.asarray(n)).astype(np.float32)).cuda()
    a = torch.from_numpy((true_a * 0.8).astype(np.complex64)).cuda()
    err0 = np.abs(f.cpu().numpy() - true_f) * np.asarray(n)
    R.rsft_refine(plan, x, k, f, a, 20, 0.7)
    torch.cuda.synchronize()
    err1 = np.abs(f.cpu().numpy() - true_f) * np.asarray(n)
    rmse0, rmse1 = math.sqrt(np.mean(err0 ** 2)), math.sqrt(np.mean(err1 ** 2))
    assert rmse1 < 0.1 * rmse0, (rmse0, rmse1)
    assert np.max(np.abs(a.cpu().numpy() - true_a) / np.abs(true_a)) < 0.05


def test_refinement_keeps_only_steps_that_lower_the_loss():
    """Two tones 1.5 bins apart with a third model tone on the same pair: the per-tone steps are
    coupled, so single trials can raise the loss; the iteration keeps only trials that lower it,
    ends at the best kept point, and zero steps leave the tones as given."""
    n, b, loops = (64, 64), (8, 8), 6
    true_f = np.array([[20.3, 30.6], [21.8, 30.9]]) / 64.0
    true_a = np.array([1.5 + 0.5j, -1.0 + 1.2j])
    rng = np.random.default_rng(8)
    cube = O.tone_field(n, true_f, true_a) + 0.05 * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
    plan = R.rsft_plan_create(R.make_desc(n, b, loops, seed=8, atten_db=50.0, p_fa1=0.05, mu=1))
    x = torch.from_numpy(cube.astype(np.complex64)).cuda()
    f0 = (np.array([[20.0, 31.0], [22.0, 31.0], [21.0, 30.0]]) / 64.0).astype(np.float32)
    a0 = np.array([1.0, 1.0j, 0.5], dtype=np.complex64)
    R.rsft_refine_prepare(plan, x)
    e_start = _eval(plan, f0, a0)[0]
    f = torch.from_numpy(f0).cuda()
    a = torch.from_numpy(a0).cuda()
    R.rsft_refine(plan, x, 3, f, a, 0, 1.0)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(f.cpu().numpy(), f0)
    np.testing.assert_array_equal(a.cpu().numpy(), a0)
    losses = [e_start]
    for steps in (1, 3, 10, 30):
        f = torch.from_numpy(f0).cuda()
        a = torch.from_numpy(a0).cuda()
        R.rsft_refine(plan, x, 3, f, a, steps, 1.0)
        torch.cuda.synchronize()
        losses.append(_eval(plan, f.cpu().numpy(), a.cpu().numpy())[0])
    assert all(l1 <= l0 for l0, l1 in zip(losses, losses[1:])), losses
    assert losses[-1] < 0.5 * losses[0], losses


def test_growing_the_tone_count_on_one_plan():
    """Evaluations with 2, then 40, then 2 tones on one plan equal those of fresh plans (the
    per-tone buffers are regrown in between)."""
    n, b, loops, tf, ta = CASES[2][1:]
    plan, x, _, f0, a0, _ = _setup(n, b, loops, np.asarray(tf), np.asarray(ta), 0.05, 6, 0.2 / np.asarray(n))
    rng = np.random.default_rng(2)
    f40 = rng.uniform(0, 1, (40, 2)).astype(np.float32)
    a40 = (rng.standard_normal(40) + 1j * rng.standard_normal(40)).astype(np.complex64)
    first = _eval(plan, f0, a0)
    many = _eval(plan, f40, a40)
    again = _eval(plan, f0, a0)
    for r0, r1 in zip(first, again):
        np.testing.assert_array_equal(np.asarray(r0), np.asarray(r1))
    fresh, _, _, _, _, _ = _setup(n, b, loops, np.asarray(tf), np.asarray(ta), 0.05, 6, 0.2 / np.asarray(n))
    for r0, r1 in zip(many, _eval(fresh, f40, a40)):
        np.testing.assert_array_equal(np.asarray(r0), np.asarray(r1))
