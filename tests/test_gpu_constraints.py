"""Parity of sph_enforce_constraints (the algebraic-constraint map after filtering, Sec. II.C) with
the oracle, through the C ABI, on a GB300.

Tolerance 1e-13 absolute on h (values of order 0.1 to 1) and 1e-13 relative to the largest |A| on
A: the map is a few dozen FP64 operations per point, the oracle and the kernel round them in a
different order (the oracle inverts the rescaled metric with numpy, the kernel divides cofactors
of the original one), and a swapped component, sign or branch gives errors of order 1e-2 or more.
Which form a point takes is an exact comparison of the same FP64 inputs on both sides.
"""
import numpy as np
import pytest

from oracle import constraints as C

pytestmark = pytest.mark.gpu

H = [1, 3, 5, 7, 9, 11]
A = [2, 4, 6, 8, 10, 12]
ALPHA = 13
NVARS = 15  # fields 0 and 14 are not touched


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_01537_gb300 import build as B
    B.build()
    return torch


def make_state(Nr, Nth, Nph, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((NVARS, Nr, Nth, Nph))
    x[H] *= 0.05  # a physical metric: det(delta + h) stays near 1
    x[ALPHA] = rng.uniform(0.0, 0.6, (Nr, Nth, Nph))
    x[ALPHA, 0, 0, 0] = 0.3  # the threshold itself: standard form
    x[ALPHA, 0, 0, -1] = 0.1  # below it, in a flagged shell: modified form
    flags = (rng.uniform(size=Nr) < 0.5).astype(np.uint8)
    flags[0] = 1
    return x, flags


def reference(x, flags):
    Nr = x.shape[1]
    fl = np.broadcast_to(flags.astype(bool)[:, None, None], x.shape[1:]) if flags is not None else False
    h2, a2 = C.enforce(x[H], x[A], x[ALPHA], fl)
    y = x.copy()
    y[H] = h2
    y[A] = a2
    return y


@pytest.mark.parametrize("shape", [(1, 1, 2), (3, 4, 8), (7, 16, 32), (5, 64, 128), (2, 97, 130)])
@pytest.mark.parametrize("with_flags", [True, False])
def test_parity(torch_cuda, shape, with_flags):
    from paper_2305_01537_gb300 import enforce_constraints
    torch = torch_cuda
    x, flags = make_state(*shape, seed=sum(shape) + with_flags)
    ref = reference(x, flags if with_flags else None)
    xd = torch.from_numpy(x).cuda()
    fd = torch.from_numpy(flags).cuda() if with_flags else None
    enforce_constraints(xd, H, A, ALPHA, fd, 0.3)
    y = xd.cpu().numpy()
    assert np.array_equal(y[[0, 14, ALPHA]], x[[0, 14, ALPHA]])
    assert np.abs(y[H] - ref[H]).max() <= 1e-13
    assert np.abs(y[A] - ref[A]).max() <= 1e-13 * np.abs(ref[A]).max()
    if with_flags:
        bh = flags.astype(bool)[:, None, None] & (x[ALPHA] < 0.3)
        # the modified form keeps A and h_12 ... h_33 bit for bit
        assert np.array_equal(y[A][:, bh], x[A][:, bh]) and np.array_equal(y[H[1:]][:, bh], x[H[1:]][:, bh])
        assert bh.any() and (~bh).any()


def test_full_size_sampled(torch_cuda):
    """128 x 64 x 128 planes (the filter's headline grid), checked on every point of a few shells."""
    from paper_2305_01537_gb300 import enforce_constraints
    torch = torch_cuda
    x, flags = make_state(128, 64, 128, seed=99)
    xd = torch.from_numpy(x).cuda()
    enforce_constraints(xd, H, A, ALPHA, torch.from_numpy(flags).cuda(), 0.3)
    y = xd.cpu().numpy()
    for i in (0, 1, 63, 127):
        xs = x[:, i:i + 1]
        ref = reference(xs, flags[i:i + 1])
        assert np.abs(y[H, i:i + 1] - ref[H]).max() <= 1e-13
        assert np.abs(y[A, i:i + 1] - ref[A]).max() <= 1e-13 * np.abs(ref[A]).max()


def test_values_outside_the_pair_range(torch_cuda):
    """Points with a value the compensated FP32 pairs cannot hold to full relative precision (tiny
    metric perturbations, huge curvature) take the FP64 path; the others the pairs. Both agree with
    the oracle point by point."""
    from paper_2305_01537_gb300 import enforce_constraints
    torch = torch_cuda
    x, flags = make_state(4, 8, 16, seed=123)
    x[H[1], 0, :2] = 1e-30        # below the pairs' range
    x[A[3], 1, :3] = 3e13         # above it
    x[A[0], 2, 0, 0] = 0.0        # zero stays on the pair path
    ref = reference(x, None)
    xd = torch.from_numpy(x).cuda()
    enforce_constraints(xd, H, A, ALPHA, None, 0.3)
    y = xd.cpu().numpy()
    scale_a = np.abs(ref[A]).max(axis=(1, 2, 3), keepdims=True)
    assert np.abs(y[H] - ref[H]).max() <= 1e-13
    assert (np.abs(y[A] - ref[A]) / scale_a).max() <= 1e-13
