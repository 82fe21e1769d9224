"""Planted mistakes in a copy of the oracle must be caught by the pins.

Each case rewrites one line of the oracle's source (a dropped term, a wrong
sign, index or factor), loads the result as a separate module on the CPU and
runs the same kinds of checks the pin tests use.  A mutation that passes all
checks would mean the pins leave that part of the oracle unchecked.
"""
import importlib.util
import math
import os
import types

import numpy as np
import numpy.polynomial.chebyshev as C
import pytest

from paper_1105_5481_gb300 import inputs as I

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "kpm_oracle.py")

MUTATIONS = {
    "doubling_drops_mu0": ("- mu0\n", "\n"),
    "doubling_wrong_vector": ("np.conj(nxt) * cur", "np.conj(nxt) * prev"),
    "doubling_factor_two": ("out[:, 2 * n] = 2.0 *", "out[:, 2 * n] = 1.0 *"),
    "direct_wrong_recursion": ("nxt = 2.0 * _rescaled_apply(H, a, b, cur) - prev\n            out",
                               "nxt = 2.0 * _rescaled_apply(H, a, b, cur) + prev\n            out"),
    "reverse_bond_not_conjugated": ("vals += [-h_k, -np.conj(h_k)]", "vals += [-h_k, -h_k]"),
    "hopping_sign": ("vals += [-h_k, -np.conj(h_k)]", "vals += [h_k, np.conj(h_k)]"),
    "rescale_shift_sign": ("return (H.matvec(X) - b * X) / a", "return (H.matvec(X) + b * X) / a"),
    "rescale_no_padding": ("return (emax - emin) / (2.0 - eps)", "return (emax - emin) / 2.0"),
    "jackson_off_by_one": ("((M - n + 1) * np.cos", "((M - n) * np.cos"),
    "dos_missing_two": ("s += 2.0 * g[n] * mu[n] * math.cos", "s += g[n] * mu[n] * math.cos"),
    "green_wrong_sign": ("-math.sin(n * th[k])", "math.sin(n * th[k])"),
    "thermo_missing_scale": ("w = a * math.pi * np.sin(", "w = math.pi * np.sin("),
    "dos_missing_jacobian": ("return a * x + b, f / a", "return a * x + b, f"),
    "dos_wrong_node": ("(np.arange(K) + 0.5) / K\n    x = np.cos(phase)",
                       "(np.arange(K) + 1.0) / K\n    x = np.cos(phase)"),
    "lorentz_wrong_argument": ("np.sinh(lam * (1.0 - n / M))", "np.sinh(lam * (1.0 - n / (M + 1)))"),
    "stats_biased_error": ("/ ((nv - 1) * nv))", "/ (nv * nv))"),
    "dos_many_missing_two": ("np.where(np.arange(M) == 0, 1.0, 2.0)", "1.0"),
    "exact_missing_norm": (".mean(axis=1)", ".sum(axis=1)"),
    "gershgorin_no_abs": ("np.abs(H.val[~on])", "H.val[~on].real"),
    "lanczos_no_residual": ("emax = theta[-1] + bk * abs(S[m - 1, -1])", "emax = theta[-1]"),
    "wrap_missing": ("xn = xn % L[d]", "xn = xn"),
    "plane_wave_coordinates_swapped": ("coords.append(i % Ld)\n        i = i // Ld",
                                       "coords.insert(0, i % Ld)\n        i = i // Ld"),
    "spectral_unnormalised": ("P = plane_waves(L, k) / math.sqrt(H.n)", "P = plane_waves(L, k)"),
    "spectral_amplitude_not_squared": ("W = np.abs(U.conj().T @ P) ** 2", "W = np.abs(U.conj().T @ P)"),
}


def load_mutant(name):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    mod = types.ModuleType("oracle_mutant_" + name)
    exec(compile(src.replace(old, new, 1), SRC, "exec"), mod.__dict__)
    return mod


def checks(O):
    """Pin-style checks; returns the list of failures."""
    fails = []

    def check(label, ok):
        if not ok:
            fails.append(label)

    def plane(L):
        g = np.meshgrid(*[np.cos(2 * np.pi * np.arange(l) / l) for l in L], indexing="ij")
        return np.sort((-2.0 * sum(g)).ravel())

    try:
        for L in [(7,), (3, 4, 5)]:
            H = O.lattice_hamiltonian(L)
            check("plane", np.allclose(np.linalg.eigvalsh(O.dense(H)), plane(L), atol=1e-12))
        w = I.workload("cubic_spin_L4")
        H = O.lattice_hamiltonian(w["L"], hop=w["hop"], onsite=I.onsite_disorder(1, 64, 1.0))
        A = O.dense(H)
        check("hermitian", np.abs(A - A.conj().T).max() == 0)
        lam = np.linalg.eigvalsh(A)
        gmin, gmax = O.gershgorin(H)
        check("gersh", gmin <= lam[0] and lam[-1] <= gmax)
        emin, emax, _ = O.lanczos_bounds(H, 12, I.lanczos_start(6, 64))
        check("lanczos", emin <= lam[0] + 1e-9 and lam[-1] - 1e-9 <= emax)
        a, b = O.rescale(gmin, gmax, 0.01)
        check("rescale", abs(a - (gmax - gmin) / 1.99) < 1e-15)
        x = (lam - b) / a
        ex = O.exact_moments(H, a, b, 24)
        check("exact", np.allclose(ex, [C.chebval(x, np.eye(n + 1)[n]).mean() for n in range(24)], atol=1e-12))
        v0 = math.sqrt(64) * np.eye(64)
        for f in (O.moments_direct, O.moments_doubling):
            mu, _ = f(H, a, b, v0, 24)
            check("fullbasis", np.allclose(mu, ex, atol=1e-12))
        M, K = 20, 40
        g = O.jackson_kernel(M)
        av = np.sin(np.pi * (np.arange(M) + 1) / (M + 1))
        av /= np.linalg.norm(av)
        check("jackson", np.allclose(g, [np.dot(av[: M - n], av[n:]) for n in range(M)], atol=1e-14))
        mu = np.linspace(1, -0.5, M)
        E, rho = O.dos(mu, 2.0, 0.1, K)
        xk = np.cos(np.pi * (np.arange(K) + 0.5) / K)
        c = 2 * g * mu
        c[0] = g[0] * mu[0]
        check("dos", np.allclose(E, 2.0 * xk + 0.1) and
              np.allclose(rho, C.chebval(xk, c) / (np.pi * np.sqrt(1 - xk * xk)) / 2.0, rtol=1e-12))
        # Lorentz kernel: the damped cosine series against its geometric closed form
        Ml, lam = 24, 3.0
        gl = O.lorentz_kernel(Ml, lam)
        r = math.exp(-lam / Ml)
        z = np.exp(1j * np.array([0.4, 1.3, 2.9]))
        G = lambda q: (1 - q ** Ml) / (1 - q)
        closed = 2 * ((math.exp(lam) * G(r * z) - math.exp(-lam) * G(z / r)) / (2 * math.sinh(lam))).real - 1
        nl = np.arange(Ml)
        direct = (((2.0 - (nl == 0)) * gl)[None, :] * np.cos(nl[None, :] * np.angle(z)[:, None])).sum(1)
        check("lorentz", np.allclose(direct, closed, atol=1e-10))
        # error bars: two vectors x1, x2 give the standard error |x1 - x2| / 2 exactly;
        # the mean DOS is the DOS of the mean moments
        P = np.array([np.linspace(1, -0.5, M), np.linspace(1, 0.3, M)])
        mu_m, mu_e, E2, rho_m, rho_e = O.stats(P, 2.0, 0.1, K)
        check("stderr", np.allclose(mu_e, np.abs(P[0] - P[1]) / 2, atol=1e-15))
        check("linear", np.allclose(rho_m, O.dos(P.mean(0), 2.0, 0.1, K)[1], atol=1e-12))
        # Green's function of one level x0 (undamped limit checked through a damped
        # series against its closed form): Re G from the sine series
        x0 = 0.3
        mu1 = np.cos(np.arange(Ml) * math.acos(x0))
        _, Gf = O.green(mu1, 1.0, 0.0, 16, "lorentz", lam)
        th = math.pi * (np.arange(16) + 0.5) / 16
        t0 = math.acos(x0)
        sines = lambda phi: 2 * ((math.exp(lam) * G(r * np.exp(1j * phi)) -
                                  math.exp(-lam) * G(np.exp(1j * phi) / r)) / (2 * math.sinh(lam))).imag
        Sk = 0.5 * (sines(th + t0) + sines(th - t0))
        check("green", np.allclose(Gf.real, -Sk / np.sin(th), atol=1e-9))
        # finite temperature: at beta = 0 every state is half filled and s = ln 2
        mu0 = np.zeros(8)
        mu0[0] = 1.0
        hot = O.thermo(mu0, 2.0, 0.0, 256, [0.0], 0.3, "none")[0]
        check("thermo", abs(hot[0] - 0.5) < 1e-12 and abs(hot[2] - math.log(2)) < 1e-12)
        # momentum-resolved moments: on a clean periodic lattice a grid plane wave
        # is an eigenvector with E(k) = -2 t sum_d cos k_d
        Ls = (5, 3, 4)
        Hc = O.lattice_hamiltonian(Ls, t=0.9)
        ac, bc = O.rescale(*O.gershgorin(Hc), eps=0.01)
        ks = 2 * math.pi * np.array([[1, 0, 0], [2, 1, 3], [0, 2, 1]]) / np.array(Ls)
        xs = (-1.8 * np.cos(ks).sum(axis=1) - bc) / ac
        want = np.cos(np.arange(12)[None, :] * np.arccos(xs)[:, None])
        check("spectral", np.allclose(O.spectral_exact(Hc, ac, bc, Ls, ks, 12), want, atol=1e-10))
    except Exception as e:  # a mutant that crashes is caught too
        fails.append("exception:" + type(e).__name__)
    return fails


def test_unmutated_oracle_passes_checks():
    spec = importlib.util.spec_from_file_location("oracle_copy", SRC)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    assert checks(mod) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    assert checks(load_mutant(name)), f"mutation {name} passed every pin check"
