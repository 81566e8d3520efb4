"""Back-to-back split-precision evaluations without host synchronisation.

An evaluation runs on the context's stream and on a side stream forked from it. This test
queues many evaluations with changing inputs (new contents in the same buffers) and reads each
result into its own buffer on the stream. `nof_jk` calls (single stream) and energy-only calls
are interleaved. Every result must equal, bit for bit, the one computed alone with a
synchronisation on both sides. A missing wait between the two streams shows up as a mismatch."""
import numpy as np
import pytest

import systems

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _t(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("graphs", [1, 0])
def test_pipelined_evaluations_match_isolated_ones(graphs):
    import paper_2512_13550_gb300 as nof
    sysm = systems.chain3s(22, seed=9)
    st = torch.cuda.Stream()
    ctx = nof.Context(precision=nof.PREC_SPLIT_BF16, stream=st, graphs=graphs)
    ctx.build_B(sysm.xyz, sysm.orb, sysm.aux)
    n, ng, a = ctx.sizes["nbf"], ctx.sizes["ngamma"], ctx.sizes["nact"]
    inputs = [(_t(sysm.orbitals(30 + k)), _t(sysm.gamma(40 + k))) for k in range(3)]

    # references: one at a time, synchronised
    ref = []
    for C, gam in inputs:
        torch.cuda.synchronize()
        E, g, gg = ctx.energy_grad(C, gam)
        J, K = ctx.jk(C)
        st.synchronize()
        ref.append((E.clone(), g.clone(), gg.clone(), J.clone(), K.clone()))

    # the same work queued back to back on the stream, inputs rewritten in place
    Cb, gb = torch.empty(n, n, dtype=torch.float64, device="cuda"), torch.empty(ng, dtype=torch.float64, device="cuda")
    E, g, gg = (torch.empty(1, dtype=torch.float64, device="cuda"), torch.empty(n, n, dtype=torch.float64, device="cuda"),
                torch.empty(ng, dtype=torch.float64, device="cuda"))
    order = [0, 1, 2, 1, 0, 0, 2, 2, 1, 0, 1, 2]
    outs = []
    torch.cuda.synchronize()
    with torch.cuda.stream(st):
        for it, k in enumerate(order):
            Cb.copy_(inputs[k][0])
            gb.copy_(inputs[k][1])
            if it % 4 == 3:  # J and K through the single-stream path
                J, K = ctx.jk(Cb)
                outs.append(("jk", k, J.clone(), K.clone()))
            elif it % 5 == 4:  # energy only (no gradient outputs)
                ctx.energy_grad(Cb, gb, E, grad=False)
                outs.append(("e", k, E.clone()))
            else:
                ctx.energy_grad(Cb, gb, E, g, gg)
                outs.append(("eg", k, E.clone(), g.clone(), gg.clone()))
    st.synchronize()
    for o in outs:
        r = ref[o[1]]
        if o[0] == "jk":
            assert torch.equal(o[2], r[3]) and torch.equal(o[3], r[4]), o[:2]
        elif o[0] == "e":
            assert o[2].item() == r[0].item(), o[:2]
        else:
            assert o[2].item() == r[0].item(), o[:2]
            assert torch.equal(o[3], r[1]) and torch.equal(o[4], r[2]), o[:2]
    # and the references themselves are right
    o = sysm.oracle
    from oracle import pnof
    for (C, gam), r in zip(inputs, ref):
        want = pnof.energy_and_gradients(o["B"], o["H"], C.cpu().numpy(), gam.cpu().numpy(), o["pm"], o["vnn"])
        assert abs(r[0].item() - want["E"]) < 1e-6
        assert np.max(np.abs(r[1].cpu().numpy() - want["g"])) < 1e-6
    ctx.close()
