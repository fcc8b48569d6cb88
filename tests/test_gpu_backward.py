"""GPU backward (hef_edge_resistance_backward, through the C ABI) against
central finite differences of the FP64 oracle, and exact invariants of the
derivative at full size.

Tolerance against the finite differences: 1e-4 relative on every resolved
coordinate.  A coordinate is resolved when the difference quotients with
steps h = 1e-5 w_e and 4h agree to 1e-5 (their gap bounds the quotient's own
rounding and truncation error); the others are counted, as are coordinates
whose routing changes between the two ends of a step (excluded)."""
import numpy as np
import pytest
import torch

from netlists import start_block, workload
from oracle import hef_grad as G
from tests._gpu import DEV, to_dev

pytestmark = pytest.mark.gpu

FD_TOL = 1e-4


def hef():
    import paper_2511_06600_gb300 as m
    return m


def forward_backward(H, x0c, x0b, k, dtype, g, use_tape=True, clique_mode=0):
    """GPU forward (keeping the tape) and backward for dL/dR = g."""
    h = hef()
    t = to_dev(H, x0c, x0b)
    inc = h.build_incidence(H.n, t["eptr"], t["pins"], t["w"], clique_mode)
    S = x0c.shape[1]
    K = 2 * k * S
    if use_tape:
        V, tape = h.krylov_basis_tape(inc, t["x0c"], t["x0b"], k, dtype)
    else:
        V, tape = h.krylov_basis(inc, t["x0c"], t["x0b"], k, dtype), None
    Q, Rf, rank = h.orthonormalize(V, K, want_R=True)
    sc = h.edge_resistance(inc, Q, K)
    gd = torch.from_numpy(np.asarray(g, dtype=np.float64)).to(DEV)
    dw, dxc, dxb = h.edge_resistance_backward(inc, k, t["x0c"], t["x0b"], Q, Rf, sc, gd, tape=tape)
    torch.cuda.synchronize()
    inc.check()
    return dict(R=sc["R"].cpu().numpy(), dw=dw.cpu().numpy(), dxc=dxc.cpu().numpy(),
                dxb=dxb.cpu().numpy(), rank=int(rank.item()), argvec=sc["argvec"].cpu().numpy())


def subset_weights(H, seed, frac=0.1):
    """dL/dR of L = sum over a seeded subset S of w_e R_e: g_e = w_e on S."""
    rng = np.random.default_rng(seed)
    S = rng.random(H.m) < frac
    return np.where(S, H.w, 0.0), S


def resolved_fd(H, x0c, x0b, k, g, coords, clique="hyperedge"):
    """Central differences at steps 1e-5 w_e and 4e-5 w_e; returns the first,
    and the mask of coordinates with unchanged routing at both steps whose
    two quotients agree to 1e-5 relative."""
    fd1, v1 = G.weight_gradient(H.n, H.eptr, H.pins, H.w, x0c, x0b, k, g, coords, rel_h=1e-5,
                                clique=clique)
    fd4, v4 = G.weight_gradient(H.n, H.eptr, H.pins, H.w, x0c, x0b, k, g, coords, rel_h=4e-5,
                                clique=clique)
    ok = v1 & v4
    resolved = ok & (np.abs(fd1 - fd4) <= 1e-5 * np.abs(fd1))
    return fd1, ok, resolved


@pytest.mark.parametrize("clique_mode", [0, 1])
def test_backward_weights_match_fd(clique_mode):
    H, k, S = workload("grid64x32_m2300_logw")
    x0c, x0b = start_block(H.n, H.m, S, 0)
    g, sel = subset_weights(H, 5)
    out = forward_backward(H, x0c, x0b, k, torch.float64, g, clique_mode=clique_mode)
    rng = np.random.default_rng(11)
    coords = np.concatenate([rng.choice(np.flatnonzero(sel), 32, replace=False),
                             rng.choice(np.flatnonzero(~sel), 32, replace=False)])
    clique = "paper" if clique_mode else "hyperedge"
    fd, valid, resolved = resolved_fd(H, x0c, x0b, k, g, coords, clique)
    assert valid.sum() >= 56, f"routing changed on {64 - valid.sum()} of 64 coordinates"
    assert resolved.sum() >= 48, f"only {resolved.sum()} of {valid.sum()} coordinates resolved"
    err = np.abs(out["dw"][coords][resolved] - fd[resolved]) / np.abs(fd[resolved])
    assert err.max() <= FD_TOL, (err.max(), coords[resolved][err.argmax()])


def test_fp32_backward_matches_fd():
    """The FP32 form's backward (FP32 QR and chain adjoints) against the FP64
    oracle's difference quotients on the resolved coordinates: within the
    reduced forms' 2e-3, relative to the largest gradient sampled."""
    H, k, S = workload("grid64x32_m2300_logw")
    x0c, x0b = start_block(H.n, H.m, S, 0)
    g, sel = subset_weights(H, 5)
    out = forward_backward(H, x0c, x0b, k, torch.float32, g)
    rng = np.random.default_rng(12)
    coords = np.concatenate([rng.choice(np.flatnonzero(sel), 24, replace=False),
                             rng.choice(np.flatnonzero(~sel), 24, replace=False)])
    fd, valid, resolved = resolved_fd(H, x0c, x0b, k, g, coords)
    assert resolved.sum() >= 36
    err = np.abs(out["dw"][coords][resolved] - fd[resolved]) / np.abs(fd[resolved]).max()
    assert err.max() <= 2e-3, err.max()


def test_backward_directions_match_fd():
    H, k, S = workload("grid64x32_m2300_logw")
    x0c, x0b = start_block(H.n, H.m, S, 0)
    g, _ = subset_weights(H, 5)
    out = forward_backward(H, x0c, x0b, k, torch.float64, g)
    rng = np.random.default_rng(21)
    checked = 0
    for _ in range(4):
        dw = rng.standard_normal(H.m) * H.w
        dxc = rng.standard_normal(x0c.shape)
        dxb = rng.standard_normal(x0b.shape)
        fd, ok = G.directional(H.n, H.eptr, H.pins, H.w, x0c, x0b, k, g, dw, dxc, dxb, h=1e-7)
        if not ok:
            continue
        got = out["dw"] @ dw + (out["dxc"] * dxc).sum() + (out["dxb"] * dxb).sum()
        assert abs(got - fd) <= FD_TOL * abs(fd), (got, fd)
        checked += 1
    assert checked >= 3


def invariants(H, x0c, x0b, out, g):
    """Exact identities of the derivative (see the oracle pin tests):
    Euler sum_e w_e dL/dw_e = -L; each chain's start direction and the
    constant direction carry no gradient."""
    L = float(g @ out["R"])
    euler = abs(float(H.w @ out["dw"]) + L) / L
    n = H.n
    chain = max(abs(float((x0c[:, s] * out["dxc"][:, s]).sum())) for s in range(x0c.shape[1]))
    chain = max(chain, max(abs(float((x0b[:, s] * out["dxb"][:, s]).sum()))
                           for s in range(x0b.shape[1])))
    gscale = max(np.abs(out["dxc"]).max(), np.abs(out["dxb"]).max()) * np.sqrt(n)
    const = abs(float(out["dxc"].sum(axis=0).max()))
    return euler, chain / gscale, const / gscale


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-9), (torch.float32, 2e-3)])
def test_backward_invariants_small(dtype, tol):
    H, k, S = workload("grid64x32_m2300_logw")
    x0c, x0b = start_block(H.n, H.m, S, 0)
    g, _ = subset_weights(H, 5)
    out = forward_backward(H, x0c, x0b, k, dtype, g)
    euler, chain, const = invariants(H, x0c, x0b, out, g)
    assert euler < tol and chain < tol and const < tol, (euler, chain, const)


@pytest.mark.slow
def test_backward_invariants_full_size_fp32():
    """The 500 x 400 grid with 210,000 log-uniform-weight hyperedges (k = 10,
    S = 1), FP32 form, as timed by the benchmark's backward leg."""
    H, k, S = workload("grid500x400_m210k_logw")
    x0c, x0b = start_block(H.n, H.m, S, 5)
    g, _ = subset_weights(H, 5)
    out = forward_backward(H, x0c, x0b, k, torch.float32, g)
    assert np.isfinite(out["dw"]).all()
    euler, chain, const = invariants(H, x0c, x0b, out, g)
    assert euler < 2e-3 and chain < 2e-3 and const < 2e-3, (euler, chain, const)


def test_backward_tape_equals_recompute_and_fp32_close():
    H, k, S = workload("grid64x32_m2300_logw")
    x0c, x0b = start_block(H.n, H.m, S, 0)
    g, _ = subset_weights(H, 5)
    a = forward_backward(H, x0c, x0b, k, torch.float64, g, use_tape=True)
    b = forward_backward(H, x0c, x0b, k, torch.float64, g, use_tape=False)
    scale = np.abs(a["dw"]).max()
    assert np.abs(a["dw"] - b["dw"]).max() <= 1e-12 * scale
    c = forward_backward(H, x0c, x0b, k, torch.float32, g)
    assert np.abs(c["dw"] - a["dw"]).max() <= 2e-3 * scale


def test_autograd_function_matches_direct_call():
    """HefResistance: L = sum_{e in S} w_e R_e; torch's dL/dw is the explicit
    term R_e on S plus the backward with dL/dR = w on S."""
    h = hef()
    H, k, S = workload("grid64x32_m2300_logw")
    x0c, x0b = start_block(H.n, H.m, S, 0)
    g, sel = subset_weights(H, 5)
    t = to_dev(H, x0c, x0b)
    w = t["w"].clone().requires_grad_(True)
    xc = t["x0c"].clone().requires_grad_(True)
    xb = t["x0b"].clone()
    R = h.resistance(w, xc, xb, H.n, t["eptr"], t["pins"], k)
    mask = torch.from_numpy(sel).to(DEV)
    L = (w * R * mask).sum()
    dw, dxc = torch.autograd.grad(L, [w, xc])
    ref = forward_backward(H, x0c, x0b, k, torch.float64, g)
    expect = ref["dw"] + np.where(sel, ref["R"], 0.0)
    assert np.allclose(dw.cpu().numpy(), expect, rtol=1e-10, atol=1e-14 * np.abs(expect).max())
    assert np.allclose(dxc.cpu().numpy(), ref["dxc"], rtol=1e-10,
                       atol=1e-14 * np.abs(ref["dxc"]).max())


def test_memory_plan_and_recompute_through_autograd():
    """hef_backward_plan keeps the tape when it fits the budget, else the
    backward recomputes the chains; HefResistance gives the same gradients
    both ways."""
    h = hef()
    H, k, S = workload("grid64x32_m2300_logw")
    x0c, x0b = start_block(H.n, H.m, S, 0)
    t = to_dev(H, x0c, x0b)
    inc = h.build_incidence(H.n, t["eptr"], t["pins"], t["w"])
    keep, tb = h.backward_plan(inc, k, S, torch.float64, 1)
    assert not keep and tb > 0
    keep, tb2 = h.backward_plan(inc, k, S, torch.float64, 1 << 62)
    assert keep and tb2 == tb
    keep, _ = h.backward_plan(inc, k, S, torch.float64, 0)  # half the free memory
    assert keep
    grads = []
    for budget in (0, 1):
        w = t["w"].clone().requires_grad_(True)
        xc = t["x0c"].clone().requires_grad_(True)
        R = h.resistance(w, xc, t["x0b"], H.n, t["eptr"], t["pins"], k, tape_budget=budget)
        (R * w).sum().backward()
        grads.append((w.grad.cpu().numpy(), xc.grad.cpu().numpy()))
    (a, b), (c, d) = grads
    assert np.abs(a - c).max() <= 1e-12 * np.abs(a).max()
    assert np.abs(b - d).max() <= 1e-12 * np.abs(b).max()
