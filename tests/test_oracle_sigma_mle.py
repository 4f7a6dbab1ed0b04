"""The FP64 oracle's maximum-likelihood resolution on the sigma-fit data.

The GPU sigma fit (tests/test_gpu_adjoint.py) is judged against this point:
the maximiser of the oracle's list-mode Poisson log-likelihood (the function
whose EM step is Eq. iter, with the kernel of Eq. kernel) over
(log sigma_z, log sigma_dl), on the same events, windows (5 sigma, rebuilt at
every sigma) and image (the true phantom).  This test finds it by Newton's
method on the oracle's analytic gradient and checks it against the value that
tests/golden/sigma_mle.py stored, that it is a maximum, and how far it lies
from the true resolution the events were simulated with.
"""
import importlib.util
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _mle_module():
    spec = importlib.util.spec_from_file_location(
        "sigma_mle", os.path.join(HERE, "golden", "sigma_mle.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_oracle_finds_the_stored_sigma_maximiser():
    m = _mle_module()
    w, ev, rho = m.fit_data()
    sig, g, Hm, evals = m.oracle_mle(w, ev, rho, tol=1e-6, central=False, final_hessian=False)
    gold = m.read_golden()
    assert gold["n_events"] == m.N_FIT and gold["cut"] == m.CUT
    np.testing.assert_allclose(sig, [gold["sigma_z"], gold["sigma_dl"]], rtol=1e-5)
    # a maximum: the gradient vanishes and the Hessian is negative definite
    assert np.abs(g).max() < 1e-3
    assert np.all(np.linalg.eigvalsh(Hm) < 0)
    # the model itself (Laplace kernel, acceptance left out of the kernel,
    # pixel-centre image) recovers the simulated resolution within 2% here
    assert abs(sig[0] / m.TRUTH[0] - 1) < 0.02 and abs(sig[1] / m.TRUTH[1] - 1) < 0.02
