"""Recorded-graph replay of nof_energy_grad (option graphs): the second call in a row with the same
pointers records the evaluation as a CUDA graph and later calls replay it. Replays must give the
same bits as direct launches, follow in-place changes of C and gamma, and count the same kernels."""
import numpy as np
import pytest

import systems

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GATE = 1e-6


def _t(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _ctx(nof, sysm, precision, graphs):
    ctx = nof.Context(precision=precision, stream=torch.cuda.Stream(), graphs=graphs)
    ctx.build_B(sysm.xyz, sysm.orb, sysm.aux)
    return ctx


def _eval(nof, ctx, C, gam, E, g, gg):
    l0 = nof.kernel_launches()
    ctx.energy_grad(C, gam, E, g, gg)
    ctx.stream.synchronize()
    return nof.kernel_launches() - l0


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_matches_direct_launches(precision):
    import paper_2512_13550_gb300 as nof
    from oracle import pnof
    sysm = systems.chain3s(14, seed=7)
    o = sysm.oracle
    cg, cd = _ctx(nof, sysm, precision, 1), _ctx(nof, sysm, precision, 0)
    n, ng = cg.sizes["nbf"], cg.sizes["ngamma"]
    C, gam = _t(sysm.orbitals(11)), _t(sysm.gamma(12))
    out = lambda: (torch.empty(1, dtype=torch.float64, device="cuda"),
                   torch.empty(n, n, dtype=torch.float64, device="cuda"),
                   torch.empty(ng, dtype=torch.float64, device="cuda"))
    Eg, gg_, ggg = out()
    Ed, gd, ggd = out()
    torch.cuda.synchronize()

    def same():
        assert Eg.item() == Ed.item()
        assert torch.equal(gg_, gd) and torch.equal(ggg, ggd)

    # direct, recorded, then replayed calls with unchanged pointers
    for it in range(4):
        lg = _eval(nof, cg, C, gam, Eg, gg_, ggg)
        ld = _eval(nof, cd, C, gam, Ed, gd, ggd)
        same()
        assert lg == ld > 0, (it, lg, ld)
    ref = pnof.energy_and_gradients(o["B"], o["H"], sysm.orbitals(11), sysm.gamma(12), o["pm"], o["vnn"])
    assert abs(Eg.item() - ref["E"]) < GATE
    assert np.max(np.abs(gg_.cpu().numpy() - ref["g"])) < GATE

    # the replayed graph reads the arrays: new contents in place, same pointers
    C2, gam2 = sysm.orbitals(21), sysm.gamma(22)
    C.copy_(_t(C2))
    gam.copy_(_t(gam2))
    torch.cuda.synchronize()
    for _ in range(2):
        _eval(nof, cg, C, gam, Eg, gg_, ggg)
        _eval(nof, cd, C, gam, Ed, gd, ggd)
        same()
    ref2 = pnof.energy_and_gradients(o["B"], o["H"], C2, gam2, o["pm"], o["vnn"])
    assert abs(Eg.item() - ref2["E"]) < GATE
    assert np.max(np.abs(ggg.cpu().numpy() - ref2["g_gamma"])) < GATE

    # new output pointers: a direct call, then a new recording; the old outputs stay untouched
    old = Eg.clone()
    Eg2, gg2, ggg2 = out()
    torch.cuda.synchronize()
    for _ in range(3):
        _eval(nof, cg, C, gam, Eg2, gg2, ggg2)
        assert Eg2.item() == Ed.item()
        assert torch.equal(gg2, gd) and torch.equal(ggg2, ggd)
    assert Eg.item() == old.item()

    # energy only (no gradient outputs), and back to the first pointers
    E3 = torch.empty(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    for _ in range(3):
        cg.energy_grad(C, gam, E3, grad=False)
        cg.stream.synchronize()
        assert E3.item() == Ed.item()
    for _ in range(2):
        _eval(nof, cg, C, gam, Eg, gg_, ggg)
        same()

    # profiling switches recording off; the results do not change
    cg.profile(True)
    for _ in range(3):
        _eval(nof, cg, C, gam, Eg, gg_, ggg)
        same()
    assert cg.profile_read()[1] == 3
    cg.profile(False)
    cg.close()
    cd.close()



@pytest.mark.parametrize("nsets", [2, 5])
def test_alternating_buffer_sets_replay_their_own_graphs(nsets):
    """Up to four recorded graphs are kept: a caller alternating between 2 buffer sets gets a
    graph for each; with 5 sets in turn the least recently used graph is replaced at every
    recording. Every call gives the bits of a context that launches directly, and no call writes
    another set's outputs."""
    import paper_2512_13550_gb300 as nof
    sysm = systems.chain3s(10, seed=3)
    cg, cd = _ctx(nof, sysm, 1, 1), _ctx(nof, sysm, 1, 0)
    n, ng = cg.sizes["nbf"], cg.sizes["ngamma"]
    sets = []
    for k in range(nsets):
        sets.append(dict(C=_t(sysm.orbitals(30 + k)), gam=_t(sysm.gamma(40 + k)),
                         E=torch.full((1,), float("nan"), dtype=torch.float64, device="cuda"),
                         g=torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda"),
                         gg=torch.full((ng,), float("nan"), dtype=torch.float64, device="cuda")))
    ref = []
    for st in sets:
        E, g, gg = torch.empty(1, dtype=torch.float64, device="cuda"), torch.empty_like(st["g"]), \
            torch.empty_like(st["gg"])
        _eval(nof, cd, st["C"], st["gam"], E, g, gg)
        ref.append((E.clone(), g.clone(), gg.clone()))
    for it in range(4 * nsets):
        k = it % nsets
        st = sets[k]
        launched = _eval(nof, cg, st["C"], st["gam"], st["E"], st["g"], st["gg"])
        assert launched > 0
        assert st["E"].item() == ref[k][0].item()
        assert torch.equal(st["g"], ref[k][1]) and torch.equal(st["gg"], ref[k][2])
        for j, other in enumerate(sets):  # every set holds its own results (or none yet)
            if j != k and not torch.isnan(other["E"]).item():
                assert other["E"].item() == ref[j][0].item()
    cg.close()
    cd.close()


def test_device_counter_step_can_be_captured():
    """nof_step with t == NULL (device-side ADAM counter, fixed exp(y) scaling): direct calls and
    CUDA-graph replays of one captured step give the same bits, and both follow the host-counter
    step (rounding differences only: exp(y) is scaled differently)."""
    import paper_2512_13550_gb300 as nof
    sysm = systems.h4()
    n = sysm.oracle["n"]

    def ctx_state():
        st = torch.cuda.Stream()
        ctx = nof.Context(precision=0, stream=st)
        ctx.build_B(sysm.xyz, sysm.orb, sysm.aux)
        C, g = _t(sysm.orbitals(0)), _t(sysm.gamma(1))
        m, v = torch.zeros(n, n, dtype=torch.float64, device="cuda"), torch.zeros(n, n, dtype=torch.float64,
                                                                                   device="cuda")
        out = torch.empty(3, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        return ctx, st, C, g, m, v, out

    host, dev, rep = ctx_state(), ctx_state(), ctx_state()
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg, stream=rep[1]):
        rep[0].step(rep[2], rep[3], rep[4], rep[5], rep[6], device_counter=True)
    for it in range(12):
        host[0].step(host[2], host[3], host[4], host[5], host[6])
        dev[0].step(dev[2], dev[3], dev[4], dev[5], dev[6], device_counter=True)
        cg.replay()
        torch.cuda.synchronize()
        assert torch.equal(dev[2], rep[2]) and torch.equal(dev[3], rep[3]), it
        assert torch.equal(dev[6], rep[6]), it
        np.testing.assert_allclose(dev[2].cpu().numpy(), host[2].cpu().numpy(), rtol=0, atol=1e-10)
        assert abs(dev[6][0].item() - host[6][0].item()) < 1e-10
    for c in (host, dev, rep):
        c[0].sync()  # raises if a device-side check (range of the fixed exp(y) scaling) fired
