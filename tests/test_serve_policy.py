"""Host logic of the server's sample schedule and give-up rule (no GPU)."""
import numpy as np

from paper_2010_09341_gb300.serve import Request, SamplePolicy


def _req(target=1e-4, budget=10 ** 9):
    return Request(family="genz_gauss", d=4, params=np.zeros(8), target_rel=target, budget=budget)


def _res(n_iter, I, sigma):
    return {"n_iter": n_iter, "I": I, "sigma": sigma}


def test_first_iterations_use_n_first():
    p = SamplePolicy(n_first=1 << 17, warm_iters=2)
    r = _req()
    assert p.first_n(r) == 1 << 17
    assert p.first_n(_req(budget=1000)) == 1000
    assert p.next_n(r, 1 << 17, _res(1, 1.0, 0.5)) == 1 << 17


def test_projection_rounds_up_to_a_power_of_two():
    # rel 1e-3 after 1e6 samples, target 1e-4: 1e8 needed, 9.9e7 more over 4 iterations
    p = SamplePolicy(n_first=1 << 10, n_max=1 << 30, iters_to_target=4, step_samples=1 << 30)
    n = p.next_n(_req(), 10 ** 6, _res(5, 2.0, 2e-3))
    assert n == 1 << 25  # 2.475e7 rounded up
    # never beyond what is left of the budget
    assert p.next_n(_req(budget=10 ** 6 + 5000), 10 ** 6, _res(5, 2.0, 2e-3)) == 5000


def test_iteration_cap_grows_when_few_integrals_are_active():
    p = SamplePolicy(n_first=1 << 10, n_max=1 << 20, step_samples=1 << 28)
    r, res = _req(), _res(5, 1.0, 1.0)  # needs far more than any cap
    assert p.next_n(r, 10 ** 6, res, n_active=1) == 1 << 27
    assert p.next_n(r, 10 ** 6, res, n_active=64) == 1 << 21
    assert p.next_n(r, 10 ** 6, res, n_active=10 ** 4) == 1 << 20  # n_max is the floor


def test_give_up_rule():
    p = SamplePolicy(give_up=4.0, give_up_after=6)
    r = _req(target=1e-4, budget=10 ** 9)
    # projected total 1e8 * (1e-3/1e-4)^2 = 1e10 > 4e9: hopeless, but only from iteration 6 on
    assert not p.hopeless(r, 10 ** 8, _res(5, 1.0, 1e-3))
    assert p.hopeless(r, 10 ** 8, _res(6, 1.0, 1e-3))
    # projected 3e9 < 4e9: keep going
    assert not p.hopeless(r, 3 * 10 ** 7, _res(8, 1.0, 1e-3))
    # zero variance or zero estimate never counts as hopeless
    assert not p.hopeless(r, 10 ** 8, _res(8, 1.0, 0.0))
    assert not p.hopeless(r, 10 ** 8, _res(8, 0.0, 1.0))
    # give_up <= 0 switches the rule off
    assert not SamplePolicy(give_up=0.0).hopeless(r, 10 ** 8, _res(8, 1.0, 1e-3))
