"""ens_solve_host splits large ensembles into chunks whose host<->device copies overlap the
other chunks' solves, and the second chunk's solve runs on a stream of its own beside the
first (own queue, ordering scratch and histogram).  The results must equal the device-array
solve over all N bit for bit: both layouts, one and two trajectories per thread, ragged chunk
sizes, save times, status and counters, SDE streams (each chunk's index offset)."""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("layout,tpt", [("rowmajor", 1), ("soa", 1), ("soa", 2)])
def test_chunked_host_solve_equals_device_solve_lorenz(layout, tpt):
    from paper_2304_06835_gb300 import EnsembleSolver
    s = EnsembleSolver("lorenz")
    N = (1 << 20) + 37  # two ragged chunks
    P, U, T = (np.asarray(a, np.float32) for a in workloads.lorenz_random(N, seed=61, t1=1.0))
    if layout == "soa":
        P, U, T = (np.ascontiguousarray(a.T) for a in (P, U, T))
    kw = dict(abstol=1e-5, reltol=1e-5, schedule="persistent", tpt=tpt)
    oh, sh, gh = s.solve_host(P, U, T, alg="tsit5", layout=layout, want_stats=True, **kw)
    d = lambda a: torch.tensor(a, device="cuda")
    od, sd, gd = s.solve(d(P), d(U), d(T), alg="tsit5", layout=layout, want_stats=True, **kw)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(oh, od.cpu().numpy())
    np.testing.assert_array_equal(sh, sd.cpu().numpy())
    np.testing.assert_array_equal(gh, gd.cpu().numpy())
    s.close()


def test_chunked_host_solve_sde_streams_and_saves():
    from paper_2304_06835_gb300 import EnsembleSolver
    s = EnsembleSolver("gbm")
    N = (1 << 20) + 5  # two ragged chunks
    P, U, T = (np.ascontiguousarray(np.asarray(a, np.float32).T)
               for a in workloads.gbm_random(N, seed=62))
    kw = dict(dt=1e-3, seed=77, index_offset=11, saveat=[0.25, 0.5, 1.0], layout="soa")
    oh, sh, gh = s.solve_host(P, U, T, alg="em", want_stats=True, **kw)
    d = lambda a: torch.tensor(a, device="cuda")
    od, sd, gd = s.solve(d(P), d(U), d(T), alg="em", want_stats=True, **kw)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(oh, od.cpu().numpy())
    np.testing.assert_array_equal(sh, sd.cpu().numpy())
    np.testing.assert_array_equal(gh, gd.cpu().numpy())
    s.close()
