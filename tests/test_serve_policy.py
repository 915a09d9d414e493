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


def test_array_forms_equal_the_scalar_rules():
    """The server applies the rules to all integrals at once; on random states,
    zero estimates and variances, exhausted budgets and early iterations they
    give exactly the scalar rules' answers."""
    rng = np.random.default_rng(7)
    k = 4000
    budget = rng.choice([10 ** 5, 10 ** 7, 10 ** 9], size=k).astype(np.float64)
    target = 10.0 ** rng.uniform(-5, -3, size=k)
    used = (budget * rng.uniform(0, 1.2, size=k)).astype(np.int64)
    n_iter = rng.integers(0, 12, size=k).astype(np.int32)
    I = rng.normal(0, 1, size=k)
    I[rng.uniform(size=k) < 0.05] = 0.0
    sigma = np.abs(I) * 10.0 ** rng.uniform(-6, 0, size=k)
    sigma[rng.uniform(size=k) < 0.05] = 0.0
    # projections beyond 2^63 samples: relative error above 10 against a 1e-5 target
    sigma[:50] = 10.0 * np.abs(I[:50]) + 1.0
    target[:50] = 1e-5
    n_iter[:50] = 9
    used[:50] = (budget[:50] * 0.9).astype(np.int64)
    for pol in (SamplePolicy(), SamplePolicy(adaptive=False), SamplePolicy(give_up=0.0),
                SamplePolicy(n_first=1 << 10, n_max=1 << 30, step_samples=1 << 31)):
        for n_active in (1, 37, 5000):
            nn = pol.next_n_array(budget, target, used, n_iter, I, sigma, n_active)
            hh = pol.hopeless_array(budget, target, used, n_iter, I, sigma)
            for i in list(range(50)) + list(range(50, k, 7)):
                r = _req(target=float(target[i]), budget=int(budget[i]))
                res = _res(int(n_iter[i]), float(I[i]), float(sigma[i]))
                if used[i] < budget[i]:
                    assert nn[i] == pol.next_n(r, int(used[i]), res, n_active), i
                assert hh[i] == pol.hopeless(r, int(used[i]), res), i
