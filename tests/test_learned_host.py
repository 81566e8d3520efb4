"""Host logic of the learned starting point: the pair-rotation targets taken from converged
orbitals (no GPU, no network)."""
import numpy as np
import pytest

from paper_2512_13550_gb300 import learned


def _orthonormal(n, seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, n)))
    return q


@pytest.mark.parametrize("flip", [(1, 1), (-1, 1), (1, -1), (-1, -1)])
def test_rotation_targets_recover_pair_angles_up_to_orbital_signs(flip):
    """C = C0 R with R a product of plane rotations (g, p(g)) by known angles in (-pi/2, pi/2),
    then every converged orbital's sign changed at will: the targets are the angles, whatever the
    signs (the energy does not see them), with S the metric of C0."""
    n, npair = 10, 3
    rng = np.random.default_rng(5)
    L = rng.standard_normal((n, n)) * 0.1 + np.eye(n)
    S = L @ L.T
    # C0 orthonormal in the metric S: C0^T S C0 = 1
    w, V = np.linalg.eigh(S)
    C0 = V @ np.diag(w ** -0.5) @ V.T @ _orthonormal(n, 2)
    theta = np.array([0.3, -1.1, 0.05])
    R = np.eye(n)
    for g in range(npair):
        p = learned.pair_partner(npair, g)
        c, s = np.cos(theta[g]), np.sin(theta[g])
        G = np.eye(n)
        G[g, g] = G[p, p] = c
        G[p, g] = s   # new orbital g = cos C0_g + sin C0_p
        G[g, p] = -s
        R = R @ G
    signs = np.ones(n)
    signs[0] = flip[0]
    signs[learned.pair_partner(npair, 0)] = flip[1]
    signs[1] = -flip[1]
    C = C0 @ R @ np.diag(signs)
    np.testing.assert_allclose(learned.rotation_targets(C0, C, S, npair), theta, atol=1e-12)


def test_pair_partner_is_an_involution_onto_the_weak_orbitals():
    """p(g) = 2 npair - 1 - g maps the strongly occupied orbitals 0 .. npair-1 onto the weakly
    occupied npair .. 2 npair - 1 in reverse order (the coupling of one weak orbital per pair)."""
    for npair in (1, 2, 5):
        ps = [learned.pair_partner(npair, g) for g in range(npair)]
        assert sorted(ps) == list(range(npair, 2 * npair))
        assert all(learned.pair_partner(npair, p) == g for g, p in enumerate(ps))


class _FakeContext:
    """Stands in for a Context: optimize() answers from a table keyed by the start's first element."""

    def __init__(self, answers):
        self.answers = answers
        self.calls = []

    def optimize(self, C, gamma, **params):
        key = float(C[0])
        self.calls.append((key, params))
        return dict(self.answers[key])


def test_fallback_runs_the_core_guess_only_when_the_learned_start_does_not_converge():
    """optimize_with_fallback keeps a converged learned run as it is; after a learned run that does
    not converge it runs the core guess and reports the evaluations of both runs."""
    torch = pytest.importorskip("torch")
    learned_start = (torch.tensor([1.0]), torch.tensor([0.1]))
    core_start = (torch.tensor([2.0]), torch.tensor([0.3]))
    ctx = _FakeContext({1.0: {"converged": True, "evaluations": 40, "E": -1.0},
                        2.0: {"converged": True, "evaluations": 70, "E": -1.0}})
    r, used = learned.optimize_with_fallback(ctx, learned_start, core_start, gtol=1e-4)
    assert used is learned_start and not r["fallback"] and r["evaluations"] == 40
    assert [c[0] for c in ctx.calls] == [1.0] and ctx.calls[0][1] == {"gtol": 1e-4}

    ctx = _FakeContext({1.0: {"converged": False, "evaluations": 300, "E": -0.5},
                        2.0: {"converged": True, "evaluations": 70, "E": -1.0}})
    r, used = learned.optimize_with_fallback(ctx, learned_start, core_start)
    assert used is core_start and r["fallback"] and r["converged"]
    assert r["evaluations"] == 370 and r["E"] == -1.0
    assert [c[0] for c in ctx.calls] == [1.0, 2.0]
