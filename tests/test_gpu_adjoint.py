"""Adjoint of the rollout (reverse pass through the contact law and the integrator) on the GPU.

Checked against the FP64 reference gradient (complex-step derivative of the
oracle's rollout), against finite differences of the GPU's own forward pass,
for independence of the checkpoint interval, and through torch.autograd.
"""
import numpy as np
import pytest

import oracle
from paper_1705_03850_gb300 import adjoint, dem, workloads
from _util import oracle_params

pytestmark = pytest.mark.gpu

MATS = [workloads.Material(E=2e7, nu=0.25, e=0.7, mu=0.6, rho=2500.0),
        workloads.Material(E=8e6, nu=0.25, e=0.55, mu=0.35, rho=2500.0)]


def _blocks():
    return [workloads.dense_block(6, 5, 4, seed=60, vel=0.05, spin=10.0, mat=MATS[0], floor_v=(0.0, 0.0, 0.0)),
            workloads.dense_block(5, 6, 4, seed=61, vel=0.05, spin=10.0, mat=MATS[1], floor_v=(0.0, 0.0, 0.0))]


def _context(wls):
    sim = dem.DEM([dem.desc_from_workload(wl) for wl in wls])
    cat = lambda f: np.concatenate([getattr(w, f) for w in wls])
    state = (cat("x"), cat("v"), cat("w"), cat("r"), cat("m"))
    return sim, state


def _axis(wls):
    return np.array([[(w.lo[0] + w.hi[0]) / 2, (w.lo[1] + w.hi[1]) / 2] for w in wls])


def _params(wls):
    return np.array([[w.material.E, w.material.e, w.material.mu] for w in wls])


def _gpu_grads(wls, nsteps, K):
    sim, state = _context(wls)
    sim.set_material(_params(wls)).write_state(*state)
    sim.rollout_forward(nsteps, K)
    ax = _axis(wls)
    obs = sim.observables(ax)
    g_ke = sim.rollout_adjoint(np.tile([1.0, 0.0], (len(wls), 1)), ax)
    g_ro = sim.rollout_adjoint(np.tile([0.0, 1.0], (len(wls), 1)), ax)
    return obs, g_ke, g_ro


def _oracle_grads(wl, nsteps, axis):
    P = oracle_params(wl)
    I = 0.4 * wl.m * wl.r ** 2
    g_ke, g_ro = [], []
    for p in ("E", "e", "mu"):
        o = oracle.rollout_derivative(P, wl.x, wl.v, wl.w, wl.r, wl.m, nsteps, p)
        g_ke.append(np.sum(wl.m[:, None] * o["v"] * o["dv"]) + np.sum(I[:, None] * o["w"] * o["dw"]))
        dx = o["x"][:, 0] - axis[0]
        dy = o["x"][:, 1] - axis[1]
        rho = np.hypot(dx, dy)
        k = int(np.argmax(rho))
        g_ro.append((dx[k] * o["dx"][k, 0] + dy[k] * o["dx"][k, 1]) / rho[k])
    return np.array(g_ke), np.array(g_ro)


def test_adjoint_matches_the_fp64_reference_gradient():
    wls = _blocks()
    nsteps = 40
    obs, g_ke, g_ro = _gpu_grads(wls, nsteps, K=10)
    ax = _axis(wls)
    for k, wl in enumerate(wls):
        r_ke, r_ro = _oracle_grads(wl, nsteps, ax[k])
        scale = np.abs(_params(wls)[k])
        # relative to the gradient's size in log-parameter units (d/dln p)
        a, b = g_ke[k] * scale, r_ke * scale
        assert np.abs(a - b).max() <= 2e-3 * np.abs(b).max(), (k, a, b)
        a, b = g_ro[k] * scale, r_ro * scale
        assert np.abs(a - b).max() <= 2e-3 * np.abs(b).max() + 1e-12, (k, a, b)


def test_gradient_does_not_depend_on_the_checkpoint_interval():
    wls = _blocks()
    o1, k1, r1 = _gpu_grads(wls, 30, K=5)
    o2, k2, r2 = _gpu_grads(wls, 30, K=30)
    o3, k3, r3 = _gpu_grads(wls, 30, K=7)
    assert np.array_equal(o1, o2) and np.array_equal(k1, k2) and np.array_equal(r1, r2)
    assert np.array_equal(k1, k3) and np.array_equal(r1, r3)


def test_adjoint_matches_gpu_finite_differences():
    wls = _blocks()
    nsteps = 40
    _, g_ke, _ = _gpu_grads(wls, nsteps, K=20)
    sim, state = _context(wls)
    ax = _axis(wls)
    base = _params(wls)
    for j in range(3):
        h = 1e-3 * base[:, j]
        ke = []
        for sgn in (1.0, -1.0):
            p = base.copy()
            p[:, j] += sgn * h
            sim.set_material(p).write_state(*state)
            sim.step(nsteps)
            ke.append(sim.observables(ax)[:, 0])
        fd = (ke[0] - ke[1]) / (2 * h)
        assert np.allclose(g_ke[:, j], fd, rtol=5e-2, atol=1e-3 * np.abs(g_ke[:, j]).max()), (j, g_ke[:, j], fd)


def test_autograd_function_backward_equals_the_adjoint():
    import torch
    wls = _blocks()
    sim, state = _context(wls)
    params = torch.tensor(_params(wls), dtype=torch.float64, requires_grad=True)
    ax = _axis(wls)
    obs = adjoint.rollout(params, sim, state, 30, 10, ax)
    loss = obs[:, 0].sum() + 3.0 * obs[:, 1].sum()
    loss.backward()
    ref = sim.rollout_adjoint(np.tile([1.0, 3.0], (len(wls), 1)), ax)
    assert np.allclose(params.grad.numpy(), ref, rtol=0, atol=0)
