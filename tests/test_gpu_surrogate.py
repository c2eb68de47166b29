"""GPU test of the gated surrogate pipeline at a reduced size: solver-generated training data,
training on the tensor cores, gate calibration on a validation split, inference with the
disagreement / out-of-box gate and solver fallback.

Checked: every out-of-box sample falls back; every fallback output is exactly the FP32
solver's answer for that input; the gate ranks correctly -- in-box samples it admits have a
smaller network error (against the FP64 tol-1e-10 reference) than in-box samples it sends
back.  Member disagreement does not bound the error of every unseen sample (the error
distribution has a heavy tail, so a threshold calibrated on one split admits some larger
errors on another); the rate of admitted samples above the calibrated bound and the
comparison the bench reports -- surrogate samples/s against the plain solver's at the
loosest tolerance that meets the same maximum error -- are printed, whichever way they
come out.
"""
import time

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


def test_gated_surrogate_pipeline_small():
    from paper_2304_06835_gb300 import EnsembleSolver, GatedSurrogate, SurrogateMLP
    from paper_2304_06835_gb300.surrogate import calibrate_tau, lorenz_u1
    dev = "cuda"
    s = EnsembleSolver("lorenz")
    box = workloads.surrogate_box()
    xt = torch.tensor(workloads.surrogate_inputs(131072, seed=6), dtype=torch.float32, device=dev)
    yt, st = lorenz_u1(s, xt)
    assert int(st.abs().sum()) == 0
    xv = torch.tensor(workloads.surrogate_inputs(8192, seed=60), dtype=torch.float32, device=dev)
    yv, _ = lorenz_u1(s, xv)
    net = SurrogateMLP(box, members=4, batch_max=4096, seed=2)
    yn = yt.double().cpu().numpy()
    net.set_scaling(yn.mean(0), yn.std(0))
    net.train(xt, yt, epochs=4, batch=2048, lr=2e-3)
    # bound: four times the median validation error of the member mean
    ym = net.forward(xv)
    err_v = (ym.double().mean(0) - yv.double()).abs().max(dim=1).values.cpu().numpy()
    eps = 4.0 * float(np.median(err_v))
    tau = calibrate_tau(net, xv, yv, eps)
    g = GatedSurrogate(net, s, tau)
    xi_np = workloads.surrogate_inputs(65536, seed=7, outside_share=0.05)
    xi = torch.tensor(xi_np, dtype=torch.float32, device=dev)
    y, fb, n = g.predict(xi)
    y, fb = y.clone(), fb.cpu().numpy().astype(bool)
    assert n == int(fb.sum()) and n > 0
    outside = np.any((xi_np.astype(np.float32) < box[:, 0]) | (xi_np.astype(np.float32) > box[:, 1]),
                     axis=1)
    assert np.all(fb[outside])
    # fallback rows equal the FP32 solver on the same inputs
    idx = np.flatnonzero(fb)
    xf = xi[torch.tensor(idx, device=dev)]
    P, U = xf[:, :3].contiguous(), xf[:, 3:].contiguous()
    T = torch.zeros((len(idx), 2), dtype=torch.float32, device=dev)
    T[:, 1] = 1.0
    uf, _, _ = s.solve(P, U, T, alg="tsit5", abstol=1e-6, reltol=1e-6)
    np.testing.assert_array_equal(y.cpu().numpy()[idx], uf.cpu().numpy())
    # the gate ranks: network error of admitted vs rejected in-box samples
    rng = np.random.default_rng(0)
    inbox = np.flatnonzero(~outside)
    sample = np.sort(rng.choice(inbox, 4096, replace=False))
    st_ = torch.tensor(sample, device=dev)
    ref, _ = lorenz_u1(s, xi[st_])
    net_err = (net.forward(xi[st_]).double().mean(0) - ref.double()).abs().max(dim=1).values
    net_err = net_err.cpu().numpy()
    adm = ~fb[sample]
    assert adm.any() and (~adm).any()
    assert np.median(net_err[adm]) < np.median(net_err[~adm])
    errs = (y[st_].double() - ref.double()).abs().max(dim=1).values.cpu().numpy()
    e = float(errs.max())
    print("admitted share %.3f, admitted above eps %.3f"
          % (adm.mean(), float((net_err[adm] > eps).mean())))
    sample = sample[adm]
    # the comparison with the plain solver at the same maximum error (reported, not asserted)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.predict(xi)
    torch.cuda.synchronize()
    t_sur = time.perf_counter() - t0
    Ps, Us = xi[:, :3].t().contiguous(), xi[:, 3:].t().contiguous()
    Ts = torch.zeros((2, xi.shape[0]), dtype=torch.float32, device=dev)
    Ts[1] = 1.0
    ref_all, _ = lorenz_u1(s, xi[torch.tensor(sample, device=dev)])
    for tol in (1e-2, 1e-3, 1e-4, 1e-5, 1e-6):
        o, _, _ = s.solve(Ps, Us, Ts, alg="tsit5", layout="soa", abstol=tol, reltol=tol)
        es = (o.t()[torch.tensor(sample, device=dev)].double() - ref_all.double()).abs().max().item()
        if es <= e:
            break
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.solve(Ps, Us, Ts, alg="tsit5", layout="soa", abstol=tol, reltol=tol)
    torch.cuda.synchronize()
    t_sol = time.perf_counter() - t0
    print("surrogate %.3g samples/s (max err %.3g, fallbacks %d); solver tol %g %.3g samples/s"
          % (len(xi_np) / t_sur, e, n, tol, len(xi_np) / t_sol))
    net.check()
    net.close()
