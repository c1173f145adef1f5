"""GPU parity of the Theorem-1 probe: the explicit matrix of A built by the
library's projector against the oracle's, the sketch deviations
||U^T (S^T S - I) U|| computed on the GPU (cuSOLVER, FP64) against the
oracle's numpy SVD, and the inequality the theorem's proof rests on,
||A^+ (S^T S - I) A v|| <= (s_1 / s_k) delta ||v||, on phantom images."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2411_05771_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2411_05771_gb300 import skei
    return skei


def test_explicit_matrix_matches_oracle(S):
    from paper_2411_05771_gb300.probe import explicit_matrix
    N, n_ang = 16, 24
    plan = S.Plan(N, n_ang)
    A = explicit_matrix(plan, batch=100).double().cpu().numpy()
    ref = O.explicit_matrix(N, plan.angles_deg, plan.n_det)
    assert A.shape == ref.shape
    assert np.abs(A - ref).max() <= 1e-6 * np.abs(ref).max()


def test_theorem1_deltas_and_proof_inequality(S):
    from paper_2411_05771_gb300.probe import theorem1
    N, n_ang = 16, 24
    plan = S.Plan(N, n_ang)
    v = torch.tensor(np.stack([I.rasterize(I.random_ellipses(s), N) for s in range(4)]),
                     dtype=torch.float32, device="cuda")
    res = theorem1(plan, ns_list=(2, 3, 4, 6), v=v)
    A = O.explicit_matrix(N, plan.angles_deg, plan.n_det)
    for item in res["sketches"]:
        d, s = O.sketch_gram_deviation(A, n_ang, plan.n_det, item["N_S"])
        assert abs(item["delta_max"] - d.max()) <= 1e-5 * d.max()
        assert abs(item["delta_mean"] - d.mean()) <= 1e-5 * d.mean()
        assert item["proof_chain_max_ratio"] <= 1.0 + 1e-6
    assert res["rank"] == int(np.sum(s > 1e-10 * s[0]))
    assert abs(res["kappa"] - s[0] / s[-1]) <= 1e-4 * s[0] / s[-1]
