"""GPU tests of the batched ensemble (ens_batch_*: one CUDA graph over mixed models) and of the
launch-shape autotuner (ens_autotune).

The per-trajectory arithmetic of a solve does not depend on the launch shape, the schedule,
the stream or the graph, so every batch result must equal, bit for bit, the same sub-problem
solved alone through ens_solve (itself parity-checked against the oracle in
test_gpu_parity.py); the full-size mixed batch is also checked against the oracle on samples.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


def dev(a, dt=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().double().numpy()


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def mixed_items(n_l, n_r, n_g, seed=4, tf_max=100.0):
    """The uneven batch: Lorenz adaptive Tsit5 with tf ~ U[1, tf_max], Robertson Rosenbrock23,
    GBM Euler-Maruyama; FP32 structure-of-arrays inputs (the mixed-batch workload)."""
    b = workloads.uneven_batch(n_l, n_r, n_g, seed=seed)
    lp, lu, lt = b["lorenz"]
    if tf_max != 100.0:
        lt[:, 1] = 1.0 + (lt[:, 1] - 1.0) * (tf_max - 1.0) / 99.0
    rp, ru, rt = b["robertson"]
    gp, gu, gt = b["gbm"]
    T = lambda a: dev(a.T)
    items = [
        dict(rhs="lorenz", params=T(lp), u0=T(lu), tspan=T(lt), alg="tsit5", abstol=1e-5,
             reltol=1e-5),
        dict(rhs="robertson", params=T(rp), u0=T(ru), tspan=T(rt), alg="ros23", abstol=1e-8,
             reltol=1e-4, dt0=1e-4),
        dict(rhs="gbm", params=T(gp), u0=T(gu), tspan=T(gt), alg="em", dt=1e-3, seed=12345),
    ]
    host_inputs = [(f32(lp), f32(lu), f32(lt)), (f32(rp), f32(ru), f32(rt)),
                   (f32(gp), f32(gu), f32(gt))]
    return items, host_inputs


def solo(it):
    from paper_2304_06835_gb300 import EnsembleSolver
    s = EnsembleSolver(it["rhs"])
    kw = {k: v for k, v in it.items() if k not in ("rhs", "params", "u0", "tspan", "alg")}
    out, st, stats = s.solve(it["params"], it["u0"], it["tspan"], alg=it["alg"], layout="soa",
                             want_stats=True, **kw)
    torch.cuda.synchronize()
    return host(out), st.cpu().numpy(), stats.cpu().numpy()


@pytest.mark.parametrize("mode", [dict(graph=True, autotune=True), dict(graph=True),
                                  dict(graph=False), dict(graph=False, serial=True),
                                  dict(graph=True, serial=True), dict(graph=True, fused=True),
                                  dict(graph=False, fused=True)])
def test_batch_equals_separate_solves(mode):
    from paper_2304_06835_gb300 import EnsembleBatch
    items, _ = mixed_items(3000, 600, 2000, seed=7, tf_max=20.0)
    ref = [solo(it) for it in items]
    b = EnsembleBatch(items, **mode)
    for rep in range(2):  # the plan (and its graph) is reusable
        outs = b.run()
        torch.cuda.synchronize()
        for (o, st, stats), (ro, rst, rstats) in zip(outs, ref):
            np.testing.assert_array_equal(host(o), ro)
            np.testing.assert_array_equal(st.cpu().numpy(), rst)
            np.testing.assert_array_equal(stats.cpu().numpy(), rstats)
    info = b.info()
    assert all(i["graph"] == mode.get("graph", True) for i in info)
    if mode.get("autotune"):
        assert all(i["tuned_ms"] > 0 and i["block"] in (64, 128, 256, 512) for i in info)
        pos = [i["launch_position"] for i in info]
        assert sorted(pos) == [0, 1, 2]
        # both graph forms were timed; the plan kept the faster
        c, s_ = info[0]["graph_ms_concurrent"], info[0]["graph_ms_serial"]
        assert c > 0 and s_ > 0
        assert all(i["serial"] == (s_ < c) for i in info)
    else:
        assert all(i["graph_ms_concurrent"] == 0 and i["graph_ms_serial"] == 0 for i in info)
        assert all(i["serial"] == mode.get("serial", False) for i in info)
    b.close()


def test_batch_graph_reads_current_inputs():
    """A captured plan keeps pointers, not values: new input contents are solved on replay."""
    from paper_2304_06835_gb300 import EnsembleBatch
    items, _ = mixed_items(500, 100, 300, seed=8, tf_max=5.0)
    b = EnsembleBatch(items, graph=True)
    b.run()
    first = host(b.outputs[0][0]).copy()
    items[0]["params"][1].mul_(0.5)  # halve rho in place
    b.run()
    second = host(b.outputs[0][0])
    ref = solo(items[0])[0]
    np.testing.assert_array_equal(second, ref)
    assert not np.array_equal(first, second)
    b.close()


def test_batch_with_saveat_and_empty_item():
    from paper_2304_06835_gb300 import EnsembleBatch
    items, _ = mixed_items(700, 50, 400, seed=9, tf_max=3.0)
    items[0]["saveat"] = [0.5, 1.0, 2.0]
    z = torch.empty((3, 0), dtype=torch.float32, device="cuda")
    items.append(dict(rhs="lorenz", params=z, u0=z, tspan=torch.empty((2, 0), device="cuda"),
                      alg="tsit5"))
    b = EnsembleBatch(items, graph=True)
    outs = b.run()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(host(outs[0][0]), solo(items[0])[0])
    assert outs[3][0].shape == (3, 0)
    assert b.info()[3]["launch_position"] == -1
    b.close()


def test_autotune_picks_a_valid_shape_and_changes_no_result():
    from paper_2304_06835_gb300 import EnsembleSolver
    P, U, T = workloads.lorenz_random(20000, seed=61, t1=2.0)
    s = EnsembleSolver("lorenz")
    Pd, Ud, Td = dev(P.T), dev(U.T), dev(T.T)
    ref, _, _ = s.solve(Pd, Ud, Td, alg="tsit5", layout="soa", abstol=1e-6, reltol=1e-6,
                        block=128, tpt=1)
    ref = host(ref)
    block, tpt, bps, ms = s.autotune(Pd, Ud, Td, alg="tsit5", layout="soa", abstol=1e-6,
                                     reltol=1e-6)
    assert block in (64, 128, 256, 512) and tpt in (1, 2) and bps in (0, -3, -2) and ms > 0
    out, _, _ = s.solve(Pd, Ud, Td, alg="tsit5", layout="soa", abstol=1e-6, reltol=1e-6)
    np.testing.assert_array_equal(host(out), ref)
    b2, t2, _, _ = s.autotune(Pd, Ud, Td, alg="tsit5", layout="soa", abstol=1e-6, reltol=1e-6,
                              block=256)  # a pinned block restricts the search
    assert b2 == 256


def test_batch_rejects_bad_items():
    from paper_2304_06835_gb300 import EnsembleBatch, EnsError
    items, _ = mixed_items(10, 10, 10, seed=3, tf_max=2.0)
    items[2]["alg"] = "em"
    items[0]["alg"] = "em"  # Euler-Maruyama needs the GBM model
    with pytest.raises(EnsError):
        EnsembleBatch(items)


def test_mixed_batch_full_size_sampled():
    """The uneven workload at full size, as the bench runs it: 500k Lorenz (tf ~ U[1,100]),
    200k Robertson, 300k GBM, FP32, one graph launch.  Every output equals the separate
    ens_solve of its item bit for bit; sampled trajectories are checked against the oracle:
    Lorenz with rho < 10 (non-chaotic: a tolerance-level error stays tolerance-level over
    100 time units) within 10x tol of the FP64 tol-1e-12 reference, Robertson within 10x tol
    of the same reference, GBM against the FP64 oracle on the FP32 normal stream."""
    from paper_2304_06835_gb300 import EnsembleBatch
    items, hin = mixed_items(500_000, 200_000, 300_000, seed=4)
    b = EnsembleBatch(items, graph=True, autotune=True)
    outs = b.run()
    torch.cuda.synchronize()
    for (o, st, stats), it in zip(outs, items):
        ro, rst, rstats = solo(it)
        np.testing.assert_array_equal(host(o), ro)
        np.testing.assert_array_equal(st.cpu().numpy(), rst)
        assert int((st != 0).sum()) == 0
    rng = np.random.default_rng(0)
    # Lorenz, non-chaotic subset
    P, U, T = hin[0]
    cand = np.flatnonzero(P[:, 1] < 10.0)
    idx = rng.choice(cand, 256, replace=False)
    ref, _, _ = oracle.solve("lorenz", "tsit5", P[idx], U[idx], T[idx], abstol=1e-12,
                             reltol=1e-12)
    o = host(outs[0][0]).T[idx]
    assert np.all(np.abs(o - ref) <= 10 * (1e-5 + 1e-5 * np.abs(ref)))
    # Robertson
    P, U, T = hin[1]
    idx = rng.choice(200_000, 128, replace=False)
    fine, _, _ = oracle.solve("robertson", "ros23", P[idx], U[idx], T[idx], abstol=1e-12,
                              reltol=1e-12, dt0=1e-8)
    o = host(outs[1][0]).T[idx]
    assert np.all(np.abs(o - fine) <= 10 * (1e-8 + 1e-4 * np.abs(fine)))
    # GBM: trajectory i of the item draws Philox stream i
    P, U, T = hin[2]
    idx = rng.choice(300_000, 256, replace=False)
    ref = np.array([oracle.solve("gbm", "em", P[i:i + 1], U[i:i + 1], T[i:i + 1], dt=1e-3,
                                 seed=12345, index_offset=int(i),
                                 precision="f64_f32stream")[0][0, 0] for i in idx])
    o = host(outs[2][0]).T[idx][:, 0]
    assert np.max(np.abs(o - ref) / np.maximum(np.abs(ref), 1)) <= 1e-5
    b.close()


def test_autotune_skips_shapes_that_do_not_fit():
    """Rosenbrock23 in FP64 uses too many registers for 512-thread blocks: the tuner must
    skip that shape, not fail."""
    from paper_2304_06835_gb300 import EnsembleSolver
    P, U, T = workloads.robertson_random(3000, seed=71)
    s = EnsembleSolver("robertson")
    d = lambda a: torch.tensor(np.ascontiguousarray(a.T), dtype=torch.float64, device="cuda")
    block, tpt, bps, ms = s.autotune(d(P), d(U), d(T), alg="ros23", layout="soa", abstol=1e-6,
                                     reltol=1e-6, dt0=1e-4)
    assert block in (64, 128, 256, 512) and ms > 0
    assert tpt == 1  # Rosenbrock23 runs one trajectory per thread: no tpt-2 candidates
    out, st, _ = s.solve(d(P), d(U), d(T), alg="ros23", layout="soa", abstol=1e-6, reltol=1e-6,
                         dt0=1e-4)
    assert int(st.abs().sum()) == 0


def test_fused_batch_lane_slots_and_refusals():
    """The fused kernel: every item solved as alone (bit for bit), in any item order; its
    persistent loops count the lane slots they issue, so attempts / slots is each item's lane
    efficiency (<= 1); autotuning times all three forms; unsupported items are refused."""
    from paper_2304_06835_gb300 import EnsError, EnsembleBatch
    items, _ = mixed_items(4000, 800, 3000, seed=9, tf_max=30.0)
    items = [items[2], items[0], items[1]]  # GBM, Lorenz, Robertson
    ref = [solo(it) for it in items]
    b = EnsembleBatch(items, fused=True)
    outs = b.run()
    torch.cuda.synchronize()
    for (o, st, stats), (ro, rst, rstats) in zip(outs, ref):
        np.testing.assert_array_equal(host(o), ro)
        np.testing.assert_array_equal(stats.cpu().numpy(), rstats)
    for inf, (_, _, rstats) in zip(b.info(), ref):
        attempts = int(rstats[0].sum() + rstats[1].sum())
        assert inf["fused"] and inf["lane_slots"] >= attempts > 0
        print("lane efficiency %.3f" % (attempts / inf["lane_slots"]))
    b.close()
    t = EnsembleBatch(items, autotune=True)
    i0 = t.info()[0]
    assert i0["graph_ms_concurrent"] > 0 and i0["graph_ms_serial"] > 0 and i0["graph_ms_fused"] > 0
    print("graphs: concurrent %.3f serial %.3f fused %.3f ms; kept fused: %s"
          % (i0["graph_ms_concurrent"], i0["graph_ms_serial"], i0["graph_ms_fused"], i0["fused"]))
    t.close()
    with pytest.raises(EnsError):  # two Lorenz items
        EnsembleBatch([items[1], items[1]], fused=True)
    sv = dict(items[1], saveat=[0.5, 1.0])
    with pytest.raises(EnsError):  # save times
        EnsembleBatch([sv, items[2]], fused=True)
