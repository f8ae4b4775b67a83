"""The fast FP64 form's screening of the split speeds (the global Lax-Friedrichs alpha_d of
reading R2, the maximum over the cells of |u_d| + c) on the CPU.

The fast pad computes the FP64 sound speed only for cells whose FP32 estimate of |u_d| + c lies
within 2e-6 of the block's FP32 maximum and gives 0 for the others; the claim is that the block
maximum is unchanged, i.e. the cell of the exact FP64 maximum always passes the screen.  The
screen is written out here in float32 numpy, operation by operation as the kernel rounds it
(|u| and c^2 rounded to FP32, a correctly rounded FP32 square root, an FP32 sum, the threshold
m (1 - 2e-6) in FP32), over blocks of 256 cells: near-uniform states (where all speeds agree to
1e-8, the hardest case), random ones, and blocks whose maximum is shared by ties.
"""
import numpy as np

F = np.float32
TOL = F(1.0) - F(2e-6)


def _screen(ua, c2):
    """FP64 block maximum of ua + sqrt(c2) over the cells the FP32 screen keeps"""
    v32 = ua.astype(F) + np.sqrt(c2.astype(F))
    m32 = np.max(v32)
    near = ~(v32 < m32 * TOL)
    v64 = np.where(near, ua + np.sqrt(c2), 0.0)
    return np.max(v64), int(np.count_nonzero(near))


def _blocks(rng):
    for _ in range(2000):   # near-uniform: a rest state with a tiny perturbation
        c2 = 1.0 + 10.0 ** rng.uniform(-12, -3) * rng.normal(size=256)
        ua = np.abs(10.0 ** rng.uniform(-12, -3) * rng.normal(size=256))
        yield ua, c2
    for _ in range(2000):   # random speeds over several decades
        yield (np.abs(rng.normal(size=256)) * 10.0 ** rng.uniform(-3, 3),
               rng.uniform(0.1, 10.0, 256) * 10.0 ** rng.uniform(-3, 3))
    for _ in range(500):    # ties and near-ties of the maximum
        c2 = np.full(256, 1.4)
        ua = np.full(256, 0.2)
        k = rng.integers(0, 256, 3)
        ua[k] += np.array([0.0, 1e-15, 3e-16])
        yield ua, c2


def test_screened_block_maximum_is_the_exact_one():
    rng = np.random.default_rng(11)
    kept = []
    for ua, c2 in _blocks(rng):
        exact = np.max(ua + np.sqrt(c2))
        got, n = _screen(ua, c2)
        assert got == exact, (got, exact)
        kept.append(n)
    kept = np.array(kept)
    # the screen does its job on non-uniform blocks: most cells skip the FP64 square root
    assert np.median(kept[2000:4000]) < 16, np.median(kept[2000:4000])


def test_a_looser_threshold_would_lose_the_maximum():
    """without the 2e-6 margin (an exact FP32 comparison against the FP32 maximum) the cell of
    the FP64 maximum can be screened out: the margin is needed"""
    rng = np.random.default_rng(12)
    lost = 0
    for ua, c2 in _blocks(rng):
        v32 = ua.astype(F) + np.sqrt(c2.astype(F))
        near = ~(v32 < np.max(v32))
        if np.max(np.where(near, ua + np.sqrt(c2), 0.0)) != np.max(ua + np.sqrt(c2)):
            lost += 1
    assert lost > 0
