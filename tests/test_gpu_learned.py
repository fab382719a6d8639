"""GPU tests of the iterative charge solve and of the learned warm start (through the C ABI):
PCG reaches the direct projected-inverse charges and the oracle's; descriptors, MLP forward pass
and MLP gradients match the FP64 oracle; a network trained on plain-method charges cuts the PCG
iterations against a cold start at the same residual."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2509_24742_gb300 import srbe, workloads as wl

pytestmark = pytest.mark.gpu
ALPHA_A = 1.7


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def slab():
    return wl.one_shot_784()


def test_pcg_reaches_direct_and_oracle_charges(orc, slab):
    samples = orc.sample_metropolis(slab.box, slab.alpha, slab.M, slab.P, 3001, 0)
    ref = orc.System(slab, alpha_A=ALPHA_A)
    m, c = ref.modes(samples)
    ev = ref.evaluate(m, c, with_lj=False)
    with srbe.from_slab(slab, alpha_A=ALPHA_A) as ctx:
        ctx.set_k(samples)
        F0, Q0, psi0 = ctx.forces()
        ctx.set_solver(srbe.PCG, tol=1e-12, maxit=5000, warm=srbe.WARM_ZERO)
        F1, Q1, psi1 = ctx.forces()
        it, res = ctx.solver_stats()
    assert res < 1e-11 and it > 0
    assert rel(Q1, Q0) < 1e-9
    assert rel(Q1, ev["Q"]) < 1e-9
    assert abs(psi1 - psi0) < 1e-9 * abs(psi0)
    assert rel(F1, F0) < 1e-9


@pytest.mark.parametrize("tol", [1e-8, 1e-11])
def test_mixed_pcg_refinement_reaches_oracle_charges(orc, slab, tol):
    """The mixed form's PCG (FP64 iterative refinement around FP32 Jacobi-PCG) meets the FP64 residual
    bar and gives the oracle's Cholesky charges to the accuracy that residual allows."""
    samples = orc.sample_metropolis(slab.box, slab.alpha, slab.M, slab.P, 3001, 0)
    ref = orc.System(slab, alpha_A=ALPHA_A)
    m, c = ref.modes(samples)
    ev = ref.evaluate(m, c, with_lj=False)
    with srbe.from_slab(slab, precision=srbe.MIXED, alpha_A=ALPHA_A) as ctx:
        ctx.set_k(samples)
        Q0, psi0, b0 = ctx.solve_charges()
        ctx.set_solver(srbe.PCG, tol=tol, maxit=5000, warm=srbe.WARM_ZERO)
        Q1, psi1, b1 = ctx.solve_charges()
        it, res = ctx.solver_stats()
        res64 = ctx.charge_residual()
    print("mixed PCG to %.0e: %d inner FP32 iterations, relative residual %.2e (FP64 check %.2e)"
          % (tol, it, res, res64))
    assert res <= tol and res64 <= 10 * tol and it > 0
    # against the oracle's solve of the same right-hand side: the accuracy the residual allows
    Q_ref, _ = orc.cp_solve(ref.factor, slab.side, slab.dpsi, b1 * srbe.VOLT)
    assert rel(Q1, Q_ref) < 1e3 * tol
    # against the oracle's own evaluation: the mixed form's b carries FP32 rounding (~1e-6), the
    # form's charge bar
    assert rel(Q1, ev["Q"]) < 1e-5


def test_descriptors_match_oracle(slab):
    with srbe.from_slab(slab, alpha_A=ALPHA_A) as ctx:
        ctx.sample_k(1, 0)
        ctx.forces()
        D = ctx.descriptors()
    ref = omlp.descriptors(slab.box, slab.R, slab.r, slab.q, slab.rc)
    scale = np.maximum(np.abs(ref).max(0), 1e-3)
    assert np.abs((D - ref) / scale).max() < 2e-4


def test_mlp_forward_and_gradients_match_oracle(slab):
    rng = np.random.default_rng(4)
    with srbe.from_slab(slab, alpha_A=ALPHA_A) as ctx:
        ctx.mlp_init(seed=11)
        P = ctx.mlp_params().astype(np.float64)
        n_tr = omlp.N_TRAIN
        P[n_tr:n_tr + 80] = rng.normal(size=80)              # input means
        P[n_tr + 80:n_tr + 160] = rng.uniform(0.5, 2.0, 80)   # input spreads
        P[-2], P[-1] = 0.3, 0.05                              # target mean, spread
        ctx.mlp_set_params(P.astype(np.float32))
        P32 = ctx.mlp_params().astype(np.float64)
        D = rng.normal(size=(300, 80)).astype(np.float32)
        T = (0.3 + 0.05 * rng.normal(size=300)).astype(np.float32)
        y = ctx.mlp_predict(D)
        g, loss = ctx.mlp_gradients(D, T)
    y_ref = omlp.forward(P32, D.astype(np.float64))
    loss_ref, g_ref = omlp.loss_and_grad(P32, D.astype(np.float64), T.astype(np.float64))
    assert rel(y, y_ref) < 1e-5
    assert abs(loss - loss_ref) < 1e-5 * loss_ref
    o = 0
    for name, shape in omlp.SIZES[:6]:
        k = int(np.prod(shape))
        assert rel(g[o:o + k], g_ref[o:o + k]) < 1e-4, name
        o += k


def _md_small(P, M):
    return wl.make_slab("md_small", (2.0, 2.0, 12.0), 8, 8, 60, 3, alpha=3.5, eta_inv=19.79, rc=1.2, P=P, M=M,
                        dpsi_volt=1.0, seed=21, ax=0.25, ay=0.25, with_md=True)


def test_learned_warm_start_beats_cold_start():
    """With the deterministic low-k_z set only (P = 0, M = 8) b is a function of the configuration,
    so the network can learn y = A^-1 (dpsi d + b) from the descriptors.  (With P > 0 the
    random-batch part of b changes the solution by O(1) from step to step and is not a function of
    the configuration: neither the network nor the previous step predicts it.)"""
    seed = 5
    s = _md_small(0, 8)
    with srbe.from_slab(s, alpha_A=ALPHA_A, md=True) as ctx:
        ctx.minimize(50)
        Ds, Ys = [], []
        for step in range(120):                     # plain-method data: direct solve every step
            ctx.step(1, seed)
            Ds.append(ctx.descriptors())
            Ys.append(ctx.solution())
        r0, v0 = ctx.get_positions(velocities=True)
        ctx.mlp_init(seed=3)
        loss = ctx.mlp_train(np.concatenate(Ds[:100]), np.concatenate(Ys[:100]), epochs=60, batch=256, lr=2e-3,
                             weight_decay=1e-6, seed=1)
        held = np.mean([rel(ctx.mlp_predict(Ds[i]), Ys[i]) for i in range(100, 120)])
        params = ctx.mlp_params()
    assert np.isfinite(loss)
    iters = {}
    for warm in (srbe.WARM_ZERO, srbe.WARM_MODEL, srbe.WARM_PREVIOUS):
        s2 = _md_small(0, 8)
        s2.r, s2.v = r0, v0
        with srbe.from_slab(s2, alpha_A=ALPHA_A, md=True) as ctx:
            ctx.mlp_set_params(params)
            ctx.set_solver(srbe.PCG, tol=1e-8, maxit=2000, warm=warm)
            its = []
            for step in range(10):
                ctx.step(1, seed + 1)
                it, res = ctx.solver_stats()
                assert res <= 1e-8
                its.append(it)
        iters[warm] = float(np.mean(its))
    print("held-out relative error of the learned y: %.3g; PCG iterations to 1e-8: cold %.1f, learned %.1f, "
          "previous step %.1f" % (held, iters[srbe.WARM_ZERO], iters[srbe.WARM_MODEL], iters[srbe.WARM_PREVIOUS]))
    assert held < 0.5
    assert iters[srbe.WARM_MODEL] < iters[srbe.WARM_ZERO]
