"""Oracle pin of the paper's Section 4.3 observation on the second Hessian family (finite-
difference advection-diffusion source inversion): with few observations a global low-rank
approximation needs fewer Hessian-vector products than the hierarchical construction, with many
it needs more, because the global rank follows the number of observations while the H² block
ranks barely grow; both meet the tolerance (dense check at 24 x 24)."""
import numpy as np
import pytest

import oracle as O
from workloads import advdiff as AD

N_SIDE, TOL = 24, 1e-4


def _products(kappa, n_obs, global_rank):
    Z = AD.hessian_factor(N_SIDE, kappa, n_obs, 5)
    op = O.LowRankOperator(Z, 1e4)
    H = op.dense()
    h, res = O.build(op, AD.coords(N_SIDE), 16, O.ADM_STRONG, 0.7, TOL, 32, 16, 8, 256, True, 7,
                     global_rank=global_rank)
    err = np.linalg.norm(O.expand_dense(h) - H, 2) / np.linalg.norm(H, 2)
    return res.samples - res.norm_its, err, res


@pytest.mark.parametrize("kappa", [1e-1, 1e-3])
def test_global_low_rank_wins_only_with_few_observations(kappa):
    full = N_SIDE * N_SIDE - 1
    h2_few, e1, _ = _products(kappa, 16, 0)
    gl_few, e2, r_few = _products(kappa, 16, full)
    h2_many, e3, _ = _products(kappa, 256, 0)
    gl_many, e4, r_many = _products(kappa, 256, full)
    assert max(e1, e2, e3, e4) <= TOL
    assert r_few.global_passed == 1 and r_many.global_passed == 1
    assert gl_few < h2_few and gl_many > h2_many
    # the global cost follows the observations, the hierarchical one barely moves
    assert gl_many >= 5 * gl_few and h2_many <= 1.5 * h2_few
