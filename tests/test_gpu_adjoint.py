"""GPU adjoint (hps_adjoint through the C ABI and the torch.autograd.Function) against the
oracle's transposed sweeps and against central finite differences."""
import numpy as np
import pytest

import synthetic as syn
from oracle import hps
from tests.gpu_common import gpu_tree, make_case, oracle_solve, to_dev
from tests.helpers import rel_linf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_02736_gb300 import build
    build.build()


@pytest.mark.parametrize("nx,ny,p,nrhs", [(1, 1, 8, 1), (2, 2, 8, 1), (4, 4, 10, 3), (3, 2, 9, 8), (4, 2, 12, 20)])
def test_adjoint_matches_oracle(nx, ny, p, nrhs):
    from paper_1612_02736_gb300 import Solver
    case = make_case(nx, ny, p, nrhs=nrhs)
    (uc, _), ops = oracle_solve(case)
    ubar = np.random.default_rng(21).standard_normal(uc.shape)
    fb, gb, _ = hps.adjoint(case["tree"], ops, p, ubar)
    cg = hps.coeff_gradients(case["tree"], p, uc, gb)
    s = Solver(gpu_tree(case), to_dev(case["coeffs"]), p)
    u = s.solve(to_dev(case["f"]), to_dev(case["g"]))
    fbg, gbg, cgg = s.adjoint(to_dev(ubar), u=u)
    assert rel_linf(fbg.cpu().numpy(), fb) < 1e-9
    assert rel_linf(gbg.cpu().numpy(), gb) < 1e-9
    assert rel_linf(cgg.cpu().numpy(), cg) < 1e-9


def test_autograd_function_finite_differences():
    # J = 0.5 ||u - u_obs||^2; gradients from HPSFunction.backward checked against central
    # differences of J computed with GPU forward solves (h = 1e-6, rebuild each time).
    import torch
    from paper_1612_02736_gb300 import HPSFunction
    case = make_case(4, 4, 10)
    p = case["p"]
    prob = syn.VarCoeffProblem()
    c_obs = np.array(prob.coeffs(case["X"], case["Y"], perturbed=True))
    t = gpu_tree(case)
    f = to_dev(case["f"][:, 0])
    g = to_dev(case["g"][..., 0])
    u_obs = HPSFunction.apply(to_dev(c_obs), f, g, t, p).detach()

    def J(c, gg):
        u = HPSFunction.apply(c, f, gg, t, p)
        return 0.5 * torch.sum((u - u_obs) ** 2)

    c = to_dev(case["coeffs"]).requires_grad_(True)
    gg = g.clone().requires_grad_(True)
    val = J(c, gg)
    val.backward()
    h = 1e-6
    for v in syn.smooth_directions(case["X"], case["Y"], n=3):
        vd = to_dev(v)
        fd = (J(c.detach() + h * vd, g) - J(c.detach() - h * vd, g)).item() / (2 * h)
        an = torch.sum(c.grad * vd).item()
        assert abs(fd - an) < 1e-5 * abs(an)
    vg = to_dev(syn.smooth_directions(case["X"], case["Y"], n=1, seed_offset=901, fields=1)[0][0])
    fd = (J(c.detach(), g + h * vg) - J(c.detach(), g - h * vg)).item() / (2 * h)
    an = torch.sum(gg.grad * vg).item()
    assert abs(fd - an) < 1e-5 * abs(an)


def test_config5_64x64_p16_recompute_ten_directions():
    # the adjoint workload as specified: J = 0.5 ||u - u_obs||^2 over all collocation nodes
    # for the variable-coefficient operator at 64 x 64 leaves, p = 16, u_obs the solution at
    # the perturbed c; gradients through HPSFunction with leaf operators recomputed in the
    # backward pass, checked by central differences along 10 seeded smooth directions of c
    # (unit max-norm) and one of g.  At the specified step h = 1e-6 the difference quotient
    # carries the rounding of the two solves divided by h (a few 1e-4 of the derivative on
    # some directions); at h = 1e-3 that noise is a thousand times smaller and the O(h^2)
    # truncation about 1e-6, so there the adjoint must agree to 2e-5.
    import torch
    from paper_1612_02736_gb300 import HPSFunction
    case = make_case(64, 64, 16)
    p = case["p"]
    prob = syn.VarCoeffProblem()
    c_obs = np.array(prob.coeffs(case["X"], case["Y"], perturbed=True))
    t = gpu_tree(case)
    f = to_dev(case["f"][:, 0])
    g = to_dev(case["g"][..., 0])
    u_obs = HPSFunction.apply(to_dev(c_obs), f, g, t, p).detach()

    def J(c, gg, store):
        u = HPSFunction.apply(c, f, gg, t, p, store)
        return 0.5 * torch.sum((u - u_obs) ** 2)

    c = to_dev(case["coeffs"]).requires_grad_(True)
    gg = g.clone().requires_grad_(True)
    J(c, gg, False).backward()
    dirs = []
    for v1 in syn.smooth_directions(case["X"], case["Y"], n=10, seed_offset=1100, fields=1):
        v = np.zeros_like(case["coeffs"])
        v[5] = v1[0] / np.abs(v1[0]).max()
        dirs.append((to_dev(v), None))
    vg = syn.smooth_directions(case["X"], case["Y"], n=1, seed_offset=1300, fields=1)[0][0]
    dirs.append((None, to_dev(vg / np.abs(vg).max())))
    errs = {1e-6: [], 1e-3: []}
    for vc, vgd in dirs:
        an = torch.sum(c.grad * vc).item() if vc is not None else torch.sum(gg.grad * vgd).item()
        for h in errs:
            with torch.no_grad():
                if vc is not None:
                    jp, jm = J(c.detach() + h * vc, g, True), J(c.detach() - h * vc, g, True)
                else:
                    jp, jm = J(c.detach(), g + h * vgd, True), J(c.detach(), g - h * vgd, True)
            errs[h].append(abs((jp - jm).item() / (2 * h) - an) / abs(an))
    for h, e in errs.items():
        print("config-5 central differences, h = %g: relative errors %s" % (h, ["%.1e" % x for x in e]))
    assert max(errs[1e-6]) < 2e-3, errs[1e-6]
    assert max(errs[1e-3]) < 2e-5, errs[1e-3]


def test_mixed_handle_rejects_adjoint():
    from paper_1612_02736_gb300 import HPSError, Solver
    case = make_case(2, 2, 8)
    s = Solver(gpu_tree(case), to_dev(case["coeffs"]), 8, precision="mixed")
    with pytest.raises(HPSError):
        s.adjoint(to_dev(case["g"]), u=to_dev(case["g"]))
