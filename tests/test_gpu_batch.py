"""Batched evaluation of uneven geometries (many H-chain frames in one launch sequence / one graph)."""
import numpy as np
import pytest

import oracle_pool

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


@pytest.mark.slow
def test_full_batch_of_256_frames_matches_oracle_per_instance():
    """The benchmark's batch: 256 displaced chains H8..H64 (lengths seed 3, displacements
    sigma = 0.05 bohr), split precision, evaluated by one nof_energy_grad_batch call; every
    instance's E, orbital gradient and occupation gradient against the oracle at 1e-6."""
    import paper_2512_13550_gb300 as nof
    orb, aux = inputs.basis_3s_10aux()
    sizes = [int(x) for x in inputs.batch_sizes(256, seed=3, lo=8, hi=64)]
    assert min(sizes) == 8 and max(sizes) == 64
    geoms = [inputs.displaced_chain(N, seed=4 * 1000003 + i) for i, N in enumerate(sizes)]
    jobs = [(orb, aux, xyz, inputs.random_orthogonal(3 * N, 5000 + i), inputs.random_gamma(N // 2, 6000 + i))
            for i, (N, xyz) in enumerate(zip(sizes, geoms))]
    refs = oracle_pool.frames(jobs)
    ctxs, Cs, gs, Es, Gs, GGs = [], [], [], [], [], []
    for (_, _, xyz, _, gam), (C, _, _, _) in zip(jobs, refs):
        ctx = nof.Context(precision=nof.PREC_SPLIT_BF16, stream=torch.cuda.Stream())
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
    worst = {"E": 0.0, "g": 0.0, "g_gamma": 0.0}
    for (_, E_ref, g_ref, gg_ref), E, G, GG in zip(refs, Es, Gs, GGs):
        worst["E"] = max(worst["E"], abs(E.item() - E_ref))
        worst["g"] = max(worst["g"], float(np.max(np.abs(G.cpu().numpy() - g_ref))))
        worst["g_gamma"] = max(worst["g_gamma"], float(np.max(np.abs(GG.cpu().numpy() - gg_ref))))
    print("256-frame batch vs oracle, worst max |difference|:", worst)
    for key, d in worst.items():
        assert d < GATE, key
    for c in ctxs:
        c.close()
