"""The two analytic plants that stand in for Sec. V-A's simulators (shared seeded
inputs, not the controller's arithmetic), checked against physics they must obey:
closed-form motion, mirror symmetry and Newton's second law."""
import numpy as np

from workloads import plants


def test_bicycle_straight_line_closed_form():
    """No steering, no lateral motion: the tyres carry no lateral force, so the
    heading stays, vx grows by dt Fx/m per step and the position moves along
    the heading by dt times the new vx (semi-implicit Euler)."""
    psi0, vx0, a, k = 0.7, 8.0, 0.5, 120
    x = np.array([3.0, -2.0, psi0, vx0, 0.0, 0.0])
    u = np.array([0.0, a])
    for _ in range(k):
        x = plants.bicycle_step(x, u)
    dt = plants.CAR_DT
    acc = plants.CAR_FX * a / plants.CAR_MASS
    vx = vx0 + k * dt * acc
    travelled = dt * (k * vx0 + dt * acc * k * (k + 1) / 2)
    assert x[2] == psi0 and x[4] == 0.0 and x[5] == 0.0
    assert np.isclose(x[3], vx, rtol=1e-12)
    assert np.allclose(x[:2], [3.0 + travelled * np.cos(psi0), -2.0 + travelled * np.sin(psi0)],
                       rtol=1e-12, atol=1e-12)


def test_bicycle_mirror_symmetry():
    """Steering the other way from the mirrored state gives the mirrored motion
    (y, psi, vy, omega change sign; x and vx do not)."""
    rng = np.random.default_rng(3)
    x = np.column_stack([rng.uniform(-5, 5, 50), rng.uniform(-5, 5, 50), rng.uniform(-1, 1, 50),
                         rng.uniform(2, 20, 50), rng.uniform(-1, 1, 50), rng.uniform(-0.5, 0.5, 50)])
    u = np.column_stack([rng.uniform(-0.4, 0.4, 50), rng.uniform(-1, 1, 50)])
    flip = np.array([1.0, -1.0, -1.0, 1.0, -1.0, -1.0])
    a, b = x.copy(), x * flip
    for _ in range(30):
        a = plants.bicycle_step(a, u)
        b = plants.bicycle_step(b, u * np.array([-1.0, 1.0]))
    assert np.allclose(b, a * flip, rtol=1e-12, atol=1e-12)


def test_cartpole_rest_and_mirror_symmetry():
    """The upright pole at rest with no force stays at rest; pushing the other
    way from the mirrored state gives the mirrored motion."""
    x = np.zeros(4)
    for _ in range(100):
        x = plants.cartpole_step(x, np.zeros(1))
    assert np.array_equal(x, np.zeros(4))
    rng = np.random.default_rng(5)
    s = np.column_stack([rng.uniform(-0.5, 0.5, 40), rng.uniform(-2, 2, 40),
                         rng.uniform(-2, 2, 40), rng.uniform(-2, 2, 40)])
    u = rng.uniform(-1, 1, (40, 1))
    a, b = s.copy(), -s
    for _ in range(50):
        a = plants.cartpole_step(a, u)
        b = plants.cartpole_step(b, -u)
    assert np.allclose(b, -a, rtol=1e-12, atol=1e-12)


def test_cartpole_centre_of_mass_obeys_newton():
    """The only horizontal external force is the push F, so the horizontal centre
    of mass x + (m_p l sin theta) / M accelerates at F / M: with the step's
    accelerations (velocity changes over dt),
    x_acc + m_p l (theta_acc cos theta - theta_dot^2 sin theta) / M = F / M."""
    rng = np.random.default_rng(7)
    s = np.column_stack([rng.uniform(-0.5, 0.5, 200), rng.uniform(-3, 3, 200),
                         rng.uniform(-2, 2, 200), rng.uniform(-2, 2, 200)])
    u = rng.uniform(-1, 1, (200, 1))
    n = plants.cartpole_step(s, u)
    dt = plants.BOT_DT
    th, thd = s[:, 0], s[:, 1]
    th_acc = (n[:, 1] - thd) / dt
    x_acc = (n[:, 3] - s[:, 3]) / dt
    m_p, l = plants.BOT_M_POLE, plants.BOT_HALF_LEN
    M = plants.BOT_M_CART + m_p
    lhs = x_acc + m_p * l * (th_acc * np.cos(th) - thd ** 2 * np.sin(th)) / M
    assert np.allclose(lhs, plants.BOT_FORCE * u[:, 0] / M, rtol=1e-9, atol=1e-9)
