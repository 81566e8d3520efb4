"""Batched evaluation of uneven geometries (many H-chain frames in one launch sequence / one graph)."""
import numpy as np
import pytest

from oracle import integrals, pnof, reference, ri
from paper_2512_13550_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GATE = 1e-6
SIZES = [8, 10, 14, 20, 26, 32, 12, 8]  # uneven chain lengths, even electron counts


def _frames():
    orb, aux = inputs.basis_3s_10aux()
    out = []
    for i, N in enumerate(SIZES):
        xyz = inputs.displaced_chain(N, seed=4000 + i)  # AIMD-like frames: sigma = 0.05 bohr
        S, T, V = integrals.one_electron(orb, xyz)
        B = ri.fitted_B(orb, aux, xyz)
        n = S.shape[0]
        pm = pnof.PairMap(N, 1, n)
        C = reference.orthonormal_orbitals(S, inputs.random_orthogonal(n, 100 + i))
        gam = inputs.random_gamma(pm.ngamma, 200 + i)
        ref = pnof.energy_and_gradients(B, T + V, C, gam, pm, integrals.nuclear_repulsion(xyz))
        out.append((xyz, C, gam, ref))
    return orb, aux, out


def _t(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_oracle_and_single_instances(precision):
    import paper_2512_13550_gb300 as nof
    orb, aux, frames = _frames()
    ctxs, Cs, gs, Es, Gs, GGs = [], [], [], [], [], []
    for xyz, C, gam, _ in frames:
        st = torch.cuda.Stream()
        ctx = nof.Context(precision=precision, stream=st)
        ctx.build_B(xyz, orb, aux)
        ctxs.append(ctx)
        n, ng = ctx.sizes["nbf"], ctx.sizes["ngamma"]
        Cs.append(_t(C)); gs.append(_t(gam))
        Es.append(torch.empty(1, dtype=torch.float64, device="cuda"))
        Gs.append(torch.empty(n, n, dtype=torch.float64, device="cuda"))
        GGs.append(torch.empty(ng, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    nof.energy_grad_batch(ctxs, Cs, gs, Es, Gs, GGs)
    torch.cuda.synchronize()
    for (xyz, C, gam, ref), ctx, E, G, GG, Ct, gt in zip(frames, ctxs, Es, Gs, GGs, Cs, gs):
        assert abs(E.item() - ref["E"]) < GATE
        assert np.max(np.abs(G.cpu().numpy() - ref["g"])) < GATE
        assert np.max(np.abs(GG.cpu().numpy() - ref["g_gamma"])) < GATE
        # the same instance alone gives the same bits
        E1, G1, GG1 = ctx.energy_grad(Ct, gt)
        torch.cuda.synchronize()
        assert E1.item() == E.item()
        assert torch.equal(G1, G) and torch.equal(GG1, GG)


def test_batch_captured_in_one_graph():
    import paper_2512_13550_gb300 as nof
    orb, aux, frames = _frames()
    ctxs, Cs, gs, Es = [], [], [], []
    for xyz, C, gam, _ in frames:
        ctx = nof.Context(precision=nof.PREC_SPLIT_BF16, stream=torch.cuda.Stream())
        ctx.build_B(xyz, orb, aux)
        ctxs.append(ctx)
        Cs.append(_t(C)); gs.append(_t(gam))
        Es.append(torch.zeros(1, dtype=torch.float64, device="cuda"))
    master = torch.cuda.Stream()
    nof.energy_grad_batch(ctxs, Cs, gs, Es, stream=master)  # warm-up outside the capture
    torch.cuda.synchronize()
    for E in Es:
        E.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=master):
        nof.energy_grad_batch(ctxs, Cs, gs, Es, stream=master)
    for E in Es:
        E.zero_()
    torch.cuda.synchronize()
    graph.replay()
    torch.cuda.synchronize()
    for (xyz, C, gam, ref), E in zip(frames, Es):
        assert abs(E.item() - ref["E"]) < GATE
