"""The GMRES least-squares step (K4: Givens rotations, residual estimate and
back-solve in FP64 on the device) against numpy's least-squares solver on the
Hessenberg matrix the kernels built (Saad 2003, 6.5.3: y minimises
||beta e_1 - H y||_2 and |g_{J}| equals that minimum)."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _check_cycle(c, restart):
    J, H, beta, y = c["J"], c["H"], c["beta"], c["y"]
    assert 1 <= J <= restart and H.shape == (J + 1, J)
    assert np.all(np.tril(H, -2) == 0.0)
    rhs = np.zeros(J + 1)
    rhs[0] = beta
    y_ref, *_ = np.linalg.lstsq(H, rhs, rcond=None)
    # Givens QR and LAPACK's solver are both backward stable in FP64; H is as
    # well conditioned as (I - gamma P_pi) restricted to the Krylov space
    # (cond <= (1 + gamma) / (1 - gamma) = 199 at gamma = 0.99)
    cond = np.linalg.cond(H)
    assert np.max(np.abs(y - y_ref)) <= 1e-13 * cond * max(1.0, np.max(np.abs(y_ref)))
    est_ref = np.linalg.norm(rhs - H @ y_ref)
    assert abs(c["est"] - est_ref) <= 1e-12 * beta
    # the rotations' residual estimate is the true least-squares residual of y
    assert abs(np.linalg.norm(rhs - H @ y) - est_ref) <= 1e-12 * beta


@pytest.mark.parametrize("restart", [1, 5, 30, 64])
def test_policy_eval_cycle_least_squares(restart):
    from paper_2502_14474_gb300 import MDP, capi
    mdp = synth.banded(20000, 4, 8, 500, 0.5, 0.99, seed=90 + restart, dtype=np.float32)
    h = MDP.from_csr(mdp)
    pi = torch.from_numpy(np.arange(mdp.n, dtype=np.int32) % mdp.m).cuda()
    v = torch.zeros(mdp.n, dtype=torch.float64, device="cuda")
    h.policy_eval(pi, v, tol=1e-30, restart=restart, max_iters=restart,
                  raise_on_not_converged=False)
    c = capi.mdp_last_cycle(h.h)
    assert c["J"] == restart
    _check_cycle(c, restart)
    h.close()


@pytest.mark.parametrize("cgs2", [False, True])
def test_solve_cycle_least_squares(cgs2):
    from paper_2502_14474_gb300 import MDP, capi
    mdp = synth.random_sparse(30000, 6, 12, 1.0, 0.99, seed=95, dtype=np.float32)
    h = MDP.from_csr(mdp)
    h.solve(tol=0.0, inner_rtol=1e-30, max_outer=1, max_inner=30, restart=30, cgs2=cgs2,
            raise_on_not_converged=False)
    c = capi.mdp_last_cycle(h.h)
    assert c["J"] == 30
    _check_cycle(c, 30)
    h.close()
