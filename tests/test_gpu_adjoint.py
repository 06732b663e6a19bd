"""Adjoint of the time evolution (rlb_adjoint_*): gradient of the final
p_perp-weighted v2 with respect to hotspot amplitudes and eta/s, against the
oracle's own forward-mode gradient (complex-step build of the oracle, all 41
parameters of a 32 x 32, 50-step case), against central finite differences of
the GPU forward run (FP64 and FP32 storage) and of the FP64 oracle,
independent of the checkpoint interval, and through torch.autograd."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1108_5561_gb300 as rlb  # noqa: E402
from paper_1108_5561_gb300 import adjoint as ADJ  # noqa: E402
from paper_1108_5561_gb300.inputs import hotspot_basis, hotspots  # noqa: E402

NT = os.cpu_count() or 1
NX, NY, STEPS, ETA, FLOOR = 8, 7, 4, 0.16, 10.0


def _case():
    _, amps, cen = hotspots(NX, NY, dx=0.1, n=3, seed=5, spread=0.25, mean_amp=15.0)
    basis = hotspot_basis(NX, NY, cen, dx=0.1)
    return amps, basis


def _grid(prec, eta=ETA):
    return rlb.GridParams(nx=NX, ny=NY, dx=0.1, prec=prec, eta_over_s=eta, tau0=0.4, dtau=0.0036)


def _v2(prec, amps, basis, eta=ETA):
    run = rlb.Run(_grid(prec, eta))
    run.init_grid(FLOOR + amps @ basis)
    run.step(STEPS)
    return run.observables()[1]


def _adjoint(prec, amps, basis, every, arithmetic=rlb.RLB_F64):
    run = rlb.Run(_grid(prec))
    eps0 = torch.as_tensor(FLOOR + amps @ basis, dtype=torch.float64, device="cuda")
    b = torch.as_tensor(basis, dtype=torch.float64, device="cuda")
    return ADJ.v2_gradient(run, eps0, b, STEPS, every, arithmetic=arithmetic)


def _fd(prec, amps, basis, rel_h, with_eta=True):
    fd = []
    for i in range(len(amps)):
        h = rel_h * amps[i]
        ap, am = amps.copy(), amps.copy()
        ap[i] += h
        am[i] -= h
        fd.append((_v2(prec, ap, basis) - _v2(prec, am, basis)) / (2 * h))
    fde = None
    if with_eta:
        he = rel_h * ETA
        fde = (_v2(prec, amps, basis, ETA + he) - _v2(prec, amps, basis, ETA - he)) / (2 * he)
    return np.array(fd), fde


def _taped():
    with open(os.path.join(os.path.dirname(__file__), "golden", "adjoint_taped_32x32.json")) as fh:
        return json.load(fh)


@pytest.mark.parametrize("prec,arith,tol", [(rlb.RLB_F64, rlb.RLB_F64, 1e-9), (rlb.RLB_F32, rlb.RLB_F32, 1e-5)])
def test_adjoint_matches_the_oracle_forward_gradient(prec, arith, tol):
    # tests/golden/adjoint_taped_32x32.json: dv2/dA_i (40 hotspots) and
    # dv2/d(eta/s) from the oracle run in complex arithmetic (written by
    # oracle/taped_gradient.py).  FP64 storage and arithmetic: the same
    # derivatives to rounding (measured 3e-12); FP32 storage and arithmetic:
    # the gradient of the FP32 trajectory, within 1e-5 of the largest
    # component (measured 5e-7).
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from oracle.taped_gradient import CASE, case_inputs
    rec = _taped()
    eps0, amps, basis = case_inputs()
    assert np.allclose(amps, rec["amplitudes"], rtol=1e-15, atol=0)
    g = rlb.GridParams(nx=CASE["nx"], ny=CASE["ny"], dx=CASE["dx"], prec=prec, eta_over_s=CASE["eta_over_s"],
                       tau0=CASE["tau0"], dtau=CASE["dtau"])
    run = rlb.Run(g)
    v2, gA, geta = ADJ.v2_gradient(run, torch.as_tensor(eps0.reshape(-1), dtype=torch.float64, device="cuda"),
                                   torch.as_tensor(basis, dtype=torch.float64, device="cuda"), CASE["steps"], 10,
                                   arithmetic=arith)
    ref = np.array(rec["dv2_dA"])
    scale = np.abs(ref).max()
    err_A = float(np.abs(np.asarray(gA) - ref).max() / scale)
    err_eta = float(abs(geta - rec["dv2_deta_over_s"]) / abs(rec["dv2_deta_over_s"]))
    print("adjoint vs oracle forward gradient (prec %d, arithmetic %d): amplitudes %.2e, eta/s %.2e, v2 %.2e"
          % (prec, arith, err_A, err_eta, abs(v2 / rec["v2"] - 1)))
    assert abs(v2 / rec["v2"] - 1) < (1e-12 if prec == rlb.RLB_F64 else 1e-5)
    assert err_A < tol and err_eta < 10 * tol, (err_A, err_eta)


def test_stored_oracle_gradient_is_reproduced(oracle_mod):
    # one component of the stored gradient recomputed here with the oracle in
    # complex arithmetic: the file is the oracle's
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from oracle.taped_gradient import case_inputs, derivative
    rec = _taped()
    eps0, _, _ = case_inputs()
    v2, d = derivative(eps0, np.zeros_like(eps0), 1.0, NT)
    assert v2 == pytest.approx(rec["v2"], rel=1e-13)
    assert d == pytest.approx(rec["dv2_deta_over_s"], rel=1e-10)


def test_fp64_adjoint_matches_finite_differences():
    amps, basis = _case()
    v2, gA, geta = _adjoint(rlb.RLB_F64, amps, basis, every=2)
    assert v2 == pytest.approx(_v2(rlb.RLB_F64, amps, basis), rel=1e-12)
    fd, fde = _fd(rlb.RLB_F64, amps, basis, 1e-4)
    print("fp64 adjoint", gA, geta, "fd", fd, fde)
    scale = np.abs(fd).max()
    assert np.abs(gA - fd).max() < 1e-6 * scale, (gA, fd)
    assert abs(geta - fde) < 1e-5 * abs(fde), (geta, fde)


def test_fp32_adjoint():
    # the adjoint of the FP32-storage trajectory against the FP64 adjoint, and the
    # amplitude gradients against finite differences of the FP32 forward run
    # (the eta/s effect, ~1e-9 in v2 over a usable step, is below the FP32 noise)
    amps, basis = _case()
    _, g32, e32 = _adjoint(rlb.RLB_F32, amps, basis, every=2)
    _, g64, e64 = _adjoint(rlb.RLB_F64, amps, basis, every=2)
    scale = np.abs(g64).max()
    print("fp32 adjoint", g32, e32, "fp64", g64, e64)
    assert np.abs(g32 - g64).max() < 1e-3 * scale and abs(e32 - e64) < 1e-3 * abs(e64)
    fd, _ = _fd(rlb.RLB_F32, amps, basis, 0.1, with_eta=False)
    print("fp32 fd", fd)
    assert np.abs(g32 - fd).max() < 0.03 * scale, (g32, fd)


@pytest.mark.parametrize("prec", [rlb.RLB_F64, rlb.RLB_F32])
def test_fp32_arithmetic_adjoint(prec):
    # the per-node adjoint work in FP32 against the same adjoint in FP64 on the
    # same trajectory (FP64 or FP32 storage), and against finite differences
    amps, basis = _case()
    v2a, g32, e32 = _adjoint(prec, amps, basis, every=2, arithmetic=rlb.RLB_F32)
    v2b, g64, e64 = _adjoint(prec, amps, basis, every=2, arithmetic=rlb.RLB_F64)
    assert v2a == v2b
    scale = np.abs(g64).max()
    print("fp32-arithmetic adjoint", g32, e32, "fp64", g64, e64)
    assert np.abs(g32 - g64).max() < 1e-4 * scale, (g32, g64)
    assert abs(e32 - e64) < 1e-3 * abs(e64), (e32, e64)
    if prec == rlb.RLB_F64:
        fd, _ = _fd(prec, amps, basis, 1e-4, with_eta=False)
        assert np.abs(g32 - fd).max() < 1e-4 * scale, (g32, fd)


@pytest.mark.parametrize("arith,tol", [(rlb.RLB_F64, 1e-7), (rlb.RLB_F32, 1e-4)])
def test_dot_product_with_a_random_seed(arith, tol):
    # <w, J d> with J the derivative of eps0 -> (f, ln M) after STEPS steps (FP64
    # storage), by central differences along a random direction d, against
    # <J^T w, d> from the adjoint seeded with a random w (rlb_adjoint_seed),
    # reversed through every step and the initial condition
    amps, _ = _case()
    rng = np.random.default_rng(11)
    g = _grid(rlb.RLB_F64)
    eps0 = FLOOR + amps @ _case()[1]
    d = rng.standard_normal(NX * NY)
    h = 1e-4

    def state(e):
        run = rlb.Run(g)
        run.init_grid(e)
        run.step(STEPS)
        return run.populations().cpu().numpy().copy(), run.lnM().cpu().numpy().copy()

    fp, lp = state(eps0 + h * d)
    fm, lm = state(eps0 - h * d)
    wf = rng.standard_normal(fp.shape) * np.abs(fp).max(axis=1, keepdims=True) ** -1
    wl = rng.standard_normal(lp.shape)
    lhs = float(np.sum(wf * (fp - fm)) / (2 * h) + np.sum(wl * (lp - lm)) / (2 * h))
    run = rlb.Run(g)
    e0 = torch.as_tensor(eps0, dtype=torch.float64, device="cuda")
    cks = ADJ.forward_with_checkpoints(run, e0, STEPS, 1)
    adj = ADJ.Adjoint(run, arith)
    adj.seed(torch.as_tensor(wf, device="cuda"), torch.as_tensor(wl, device="cuda"))
    ADJ.reverse_sweep(run, adj, cks, STEPS, 1)
    gd, _ = adj.ic(e0, torch.as_tensor(d[None, :], dtype=torch.float64, device="cuda"))
    rhs = float(gd[0])
    print("dot product", arith, lhs, rhs, abs(lhs - rhs) / abs(lhs))
    assert abs(lhs - rhs) < tol * abs(lhs), (lhs, rhs)


def test_adjoint_arithmetic_is_checked():
    run = rlb.Run(_grid(rlb.RLB_F32))
    with pytest.raises(rlb.RLBError):
        ADJ.Adjoint(run, rlb.RLB_BF16)


def test_adjoint_matches_oracle_finite_differences(oracle_mod):
    amps, basis = _case()
    _, gA, geta = _adjoint(rlb.RLB_F64, amps, basis, every=4)

    def v2o(a, eta=ETA):
        o = oracle_mod.Oracle(nx=NX, ny=NY, dx=0.1, eta_over_s=eta)
        f, lnM = o.init_state(FLOOR + a @ basis, NT)
        o.step(f, lnM, 0.4, 0.0036, STEPS, NT)
        return o.observables(f, lnM, NT)[1]

    fd = []
    for i in range(len(amps)):
        h = 1e-4 * amps[i]
        ap, am = amps.copy(), amps.copy()
        ap[i] += h
        am[i] -= h
        fd.append((v2o(ap) - v2o(am)) / (2 * h))
    fd = np.array(fd)
    he = 1e-4 * ETA
    fde = (v2o(amps, ETA + he) - v2o(amps, ETA - he)) / (2 * he)
    print("oracle fd", fd, fde, "adjoint", gA, geta)
    scale = np.abs(fd).max()
    assert np.abs(gA - fd).max() < 1e-6 * scale
    assert abs(geta - fde) < 1e-5 * abs(fde)  # a ~1e-11 change of v2 over the eta step


def test_checkpoint_interval_does_not_change_the_gradient():
    amps, basis = _case()
    a = _adjoint(rlb.RLB_F32, amps, basis, every=1)
    b = _adjoint(rlb.RLB_F32, amps, basis, every=3)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and a[2] == b[2]


def test_autograd_function():
    amps, basis = _case()
    run = rlb.Run(_grid(rlb.RLB_F64))
    b = torch.as_tensor(basis, dtype=torch.float64, device="cuda")
    A = torch.tensor(amps, dtype=torch.float64, requires_grad=True)
    eta = torch.tensor(ETA, dtype=torch.float64, requires_grad=True)
    F = ADJ.elliptic_flow_function()
    v2 = F.apply(A, eta, run, b, FLOOR, STEPS, 2)
    v2.backward()
    _, gA, geta = _adjoint(rlb.RLB_F64, amps, basis, every=2)
    rel = np.abs(A.grad.numpy() - gA) / np.abs(gA).max()
    print("autograd", A.grad.numpy(), eta.grad.item(), "direct", gA, geta, "rel", rel)
    # the same gradient (the initial state is summed on the device here, on the host
    # there: rounding-level differences of eps0)
    assert rel.max() < 1e-8
    assert eta.grad.item() == pytest.approx(geta, rel=1e-8)


@pytest.mark.parametrize("prec,arith,tol", [(rlb.RLB_F64, rlb.RLB_F64, 1e-10), (rlb.RLB_F32, rlb.RLB_F32, 1e-5)])
def test_step_from_a_blob_equals_load_then_step(prec, arith, tol):
    amps, basis_h = _case()
    run = rlb.Run(_grid(prec))
    eps0 = torch.as_tensor(FLOOR + amps @ basis_h, dtype=torch.float64, device="cuda")
    basis = torch.as_tensor(basis_h, dtype=torch.float64, device="cuda")
    run.init_grid(eps0)
    blob0 = run.save_state(device=True)
    run.step(1)
    f1, l1, tau1 = run.populations().clone(), run.lnM().clone(), run.tau
    adj = ADJ.Adjoint(run, arith)
    adj.seed_v2()
    adj.step(blob0)  # input read in place from the blob; the run's state stays the final one
    g_blob = adj.ic(eps0, basis)
    assert torch.equal(run.populations(), f1) and torch.equal(run.lnM(), l1) and run.tau == tau1
    adj.seed_v2()
    run.load_state(blob0)
    adj.step()
    g_load = adj.ic(eps0, basis)
    scale = max(np.abs(g_load[0]).max(), 1e-300)
    assert np.abs(g_blob[0] - g_load[0]).max() / scale < tol
    assert abs(g_blob[1] - g_load[1]) <= tol * max(abs(g_load[1]), 1e-300)
