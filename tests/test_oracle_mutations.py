"""The oracle's pins reject plausible mistakes.

Each case plants one change -- a flipped sign, a dropped term, a transposed
operand, a wrong constant or index -- in a copy of the oracle on the CPU and
checks that the pins aimed at that kind of mistake fail on the mutant while
they pass on an unchanged copy:
  * the gradient and the direct sum of the C oracle (``oracle/rpy_oracle.c``,
    compiled in a temporary directory) against central differences, the
    gradient invariants and the dense matrix;
  * the RPY pair blocks against the pins of ``test_oracle_pins.py`` (the
    quadrature of the defining integral, contact values, continuity, the
    Oseen limit, half the vorticity, symmetry and positive definiteness);
  * the single-wall blocks against the sympy derivation of ``test_wall_pins.py``;
  * the Python half (square roots, Lanczos, Philox, the roller-example
    integrator), a changed copy of ``oracle/__init__.py`` executed as a
    separate module, against the pins of both files.
The oracle's own sources are never modified and no GPU is involved."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

SRC = os.path.join(os.path.dirname(os.path.abspath(oracle.__file__)), "rpy_oracle.c")
_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)

pytestmark = pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")


def _compile(tmp_path, name, old=None, new=None):
    """Build a copy of the oracle, with `old` replaced by `new` (exactly one
    occurrence), and return its ctypes handle."""
    src = open(SRC).read()
    if old is not None:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    c = tmp_path / (name + ".c")
    so = tmp_path / (name + ".so")
    c.write_text(src)
    subprocess.run(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                    str(c), "-o", str(so), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    lib.orc_grad.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double,
                             ctypes.c_int, _i64p, ctypes.c_int64, _dp]
    lib.orc_mdot.argtypes = [ctypes.c_int64, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                             ctypes.c_int, _i64p, ctypes.c_int64, _dp, _dp]
    lib.orc_assemble.argtypes = [ctypes.c_int64, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                 ctypes.c_int, _dp]
    return lib


def _p(x):
    return None if x is None else x.ctypes.data_as(_dp)


def _grad(lib, pos, F, T, G, H, angular):
    n = pos.shape[0]
    dX = np.zeros((n, 3))
    lib.orc_grad(n, _p(pos), _p(F), _p(T), _p(G), _p(H), 1.0, 1.0, int(angular), None, n, _p(dX))
    return dX


def _mdot(lib, pos, F, T, angular):
    n = pos.shape[0]
    U = np.zeros((n, 3))
    W = np.zeros((n, 3))
    lib.orc_mdot(n, _p(pos), _p(F), _p(T), 1.0, 1.0, int(angular), 0, None, n, _p(U), _p(W))
    return U, W


def _assemble(lib, pos, angular):
    n = pos.shape[0]
    dim = (6 if angular else 3) * n
    M = np.zeros((dim, dim))
    lib.orc_assemble(n, _p(pos), 1.0, 1.0, int(angular), 0, _p(M))
    return M


def _case(seed, n=24, L=5.0):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-L / 2, L / 2, size=(n, 3))   # overlapping pairs included
    F, T, G, H = (np.ascontiguousarray(rng.standard_normal((n, 3))) for _ in range(4))
    return np.ascontiguousarray(pos), F, T, G, H


def _pins(lib, angular, seed=3):
    """The gradient and product pins of the oracle (as in test_oracle_pins),
    evaluated on `lib`: True where the pin holds."""
    pos, F, T, G, H = _case(seed)
    n = pos.shape[0]
    if not angular:
        T = H = None
    dX = _grad(lib, pos, F, T, G, H, angular)

    def L(p):
        U, W = _mdot(lib, p, F, T, angular)
        return np.sum(G * U) + (np.sum(H * W) if angular else 0.0)

    h = 1e-6
    fd = np.zeros_like(pos)
    for i in range(n):
        for k in range(3):
            pp = pos.copy()
            pp[i, k] += h
            pm = pos.copy()
            pm[i, k] -= h
            fd[i, k] = (L(pp) - L(pm)) / (2 * h)
    scale = np.abs(fd).max()
    M = _assemble(lib, pos, angular)
    U, W = _mdot(lib, pos, F, T, angular)
    y = M @ (np.concatenate([F.ravel(), T.ravel()]) if angular else F.ravel())
    direct = np.concatenate([U.ravel(), W.ravel()]) if angular else U.ravel()
    pins = {
        "central_differences": np.abs(dX - fd).max() <= 2e-7 * scale,
        "sum_zero": np.abs(dX.sum(axis=0)).max() <= 1e-13 * n * np.abs(dX).max(),
        "dense_equals_direct": np.abs(direct - y).max() <= 1e-13 * np.abs(y).max(),
    }
    if angular:
        dX2 = _grad(lib, pos, G, H, F, T, angular)
        pins["exchange"] = np.abs(dX2 - dX).max() <= 1e-13 * np.abs(dX).max()
    return pins


@pytest.mark.parametrize("angular", [False, True])
def test_unchanged_copy_passes_every_pin(tmp_path, angular):
    pins = _pins(_compile(tmp_path, "same"), angular)
    assert all(pins.values()), pins


MUTATIONS = [
    # the source-role term of the chain rule added with the wrong sign
    ("sign_of_source_term", "acc[c] += sgn * s;", "acc[c] += s;", False,
     {"central_differences", "sum_zero"}),
    # the H.wF.F coupling term of the gradient dropped
    ("dropped_coupling_term", "if (H) s += H[3 * k + p] * dwF[9 * c + 3 * p + q] * F[3 * l + q];", "", True,
     {"central_differences", "exchange"}),
    # the derivative of the u-from-T block transposed
    ("transposed_coupling_derivative", "duT[9 * c + 3 * p + q]", "duT[9 * c + 3 * q + p]", True,
     {"central_differences", "exchange"}),
    # the u-from-T block transposed in the direct sum only
    ("transposed_block_in_direct_sum", "if (T) u[p] += uT[3 * p + q] * T[3 * j + q];",
     "if (T) u[p] += uT[3 * q + p] * T[3 * j + q];", True, {"central_differences", "dense_equals_direct"}),
    # the column particle of the source-role term taken from the wrong index
    ("wrong_column_particle", "const int64_t l = side == 0 ? j : i;", "const int64_t l = j;", False,
     {"central_differences"}),
]


@pytest.mark.parametrize("name,old,new,angular,caught_by", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_its_pins(tmp_path, name, old, new, angular, caught_by):
    pins = _pins(_compile(tmp_path, name, old, new), angular)
    failed = {k for k, ok in pins.items() if not ok}
    assert caught_by <= failed, (name, pins)


# --------------------------------------------------------------------------
# Pair-block mistakes, caught by the pins of test_oracle_pins run unchanged
# against the mutant (the oracle module pointed at the mutant's library).
# --------------------------------------------------------------------------
import test_oracle_pins as P  # noqa: E402

BLOCK_PINS = {
    "quadrature": lambda o: [P.test_pair_blocks_match_envelope_quadrature(o, s)
                             for s in (0.3, 1.2, 1.9, 2.05, 2.15, 3.0, 6.0)],
    "contact_golden": P.test_contact_values_golden,
    "continuous_at_contact": P.test_blocks_continuous_at_contact,
    "oseen_limit": P.test_oseen_limit,
    "half_vorticity": P.test_far_field_rotation_is_half_vorticity,
    "symmetric_positive_definite": lambda o: P.test_grand_mobility_symmetric_positive_definite(o, 40, 6.0),
    "gradient_central_differences": lambda o: P.test_gradient_matches_central_differences(o, True),
}


def _block_pins(monkeypatch, lib_path):
    monkeypatch.setattr(oracle, "_LIB_PATH", str(lib_path))
    monkeypatch.setattr(oracle, "_lib", None)
    oracle._load()
    held = {}
    for name, pin in BLOCK_PINS.items():
        try:
            pin(oracle)
            held[name] = True
        except AssertionError:
            held[name] = False
    return held


def test_unchanged_copy_passes_every_block_pin(tmp_path, monkeypatch):
    _compile(tmp_path, "same")
    held = _block_pins(monkeypatch, tmp_path / "same.so")
    assert all(held.values()), held


BLOCK_MUTATIONS = [
    # the a^2 / (3 r^3) term of the far-field tt identity coefficient without its 1/3
    ("far_field_a2_term", "c[0] = k8 * (1.0 / r + 2.0 * a * a / (3.0 * r3));", "c[0] = k8 * (1.0 / r + 2.0 * a * a / r3);",
     {"quadrature", "continuous_at_contact"}),
    # a wrong constant in the overlapping rr coefficient (the golden contact
    # values sit at r = 2a, on the far-field branch, so they cannot see it)
    ("overlap_rr_constant", "c[3] = kr * (1.0 - 27.0 * s / 32.0 + 5.0 * s * s * s / 64.0);",
     "c[3] = kr * (1.0 - 9.0 * s / 32.0 + 5.0 * s * s * s / 64.0);", {"quadrature", "continuous_at_contact"}),
    # the far-field translation-rotation coupling with the wrong sign
    ("coupling_sign", "c[2] = -k8 / r2;", "c[2] = k8 / r2;", {"half_vorticity", "continuous_at_contact"}),
    # omega-from-F block with the opposite sign of u-from-T (M no longer symmetric)
    ("rt_block_sign", "wF[3 * p + q] = c[2] * ex[3 * p + q];", "wF[3 * p + q] = -c[2] * ex[3 * p + q];",
     {"symmetric_positive_definite"}),
    # a wrong constant in the derivative of the far-field tt dd coefficient
    ("far_field_derivative", "dc[1] = k8 * (-1.0 / r2 + 6.0 * a * a / r4);", "dc[1] = k8 * (-1.0 / r2 + 2.0 * a * a / r4);",
     {"gradient_central_differences"}),
]


@pytest.mark.parametrize("name,old,new,caught_by", BLOCK_MUTATIONS, ids=[m[0] for m in BLOCK_MUTATIONS])
def test_planted_block_mistake_fails_its_pins(tmp_path, monkeypatch, name, old, new, caught_by):
    _compile(tmp_path, name, old, new)
    held = _block_pins(monkeypatch, tmp_path / (name + ".so"))
    failed = {k for k, ok in held.items() if not ok}
    assert caught_by <= failed, (name, held)


# --------------------------------------------------------------------------
# Single-wall mistakes, caught by the wall pins (the sympy derivation of the
# blocks from the Blake image system, the Swan-Brady self mobilities).
# --------------------------------------------------------------------------
import functools  # noqa: E402

import test_wall_pins as WP  # noqa: E402

_blake = functools.lru_cache(maxsize=None)(WP._blake_blocks)   # independent of the oracle

WALL_PINS = {
    "blake_definition": WP.test_wall_blocks_match_blake_definition,
    "swan_brady_self": lambda: WP.test_wall_self_mobility_matches_swan_brady(1.0, 1.0),
    "symmetric_positive_definite": lambda: WP.test_wall_matrix_symmetric_positive_definite(True),
}


def _wall_pins(monkeypatch, lib_path):
    monkeypatch.setattr(oracle, "_LIB_PATH", str(lib_path))
    monkeypatch.setattr(oracle, "_lib", None)
    monkeypatch.setattr(WP, "_blake_blocks", _blake)
    oracle._load()
    held = {}
    for name, pin in WALL_PINS.items():
        try:
            pin()
            held[name] = True
        except AssertionError:
            held[name] = False
    return held


def test_unchanged_copy_passes_every_wall_pin(tmp_path, monkeypatch):
    pytest.importorskip("sympy")
    _compile(tmp_path, "same")
    held = _wall_pins(monkeypatch, tmp_path / "same.so")
    assert all(held.values()), held


WALL_MUTATIONS = [
    # a wrong constant in the a^4 term of the tangential uF entry
    ("uF_a4_constant", "a4 * (-70.0 * c4 / 3.0 + 70.0 * c2 / 3.0 - 8.0 / 3.0) * r5",
     "a4 * (-70.0 * c4 / 3.0 + 70.0 * c2 / 3.0 - 4.0 / 3.0) * r5", {"blake_definition"}),
    # a wrong constant in the normal-normal wT entry
    ("wT_constant", "LwT[4] = (3.5 - 6.0 * c2) * r3;", "LwT[4] = (3.5 - 4.5 * c2) * r3;", {"blake_definition"}),
    # a flipped sign in the uT block
    ("uT_sign", "LuT[5] = -s * r2;", "LuT[5] = s * r2;", {"blake_definition"}),
]


@pytest.mark.parametrize("name,old,new,caught_by", WALL_MUTATIONS, ids=[m[0] for m in WALL_MUTATIONS])
def test_planted_wall_mistake_fails_its_pins(tmp_path, monkeypatch, name, old, new, caught_by):
    pytest.importorskip("sympy")
    _compile(tmp_path, name, old, new)
    held = _wall_pins(monkeypatch, tmp_path / (name + ".so"))
    failed = {k for k, ok in held.items() if not ok}
    assert caught_by <= failed, (name, held)


# --------------------------------------------------------------------------
# Mistakes in the Python half of the oracle (square roots, Lanczos, Philox,
# the roller-example integrator): a changed copy of oracle/__init__.py is
# executed as a separate module (same C library) and the pins run against it.
# --------------------------------------------------------------------------
import types  # noqa: E402

import test_integrator_pins as IP  # noqa: E402

PY_SRC = os.path.join(os.path.dirname(os.path.abspath(oracle.__file__)), "__init__.py")


def _py_mutant(old=None, new=None):
    src = open(PY_SRC).read()
    if old is not None:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    mod = types.ModuleType("oracle_mutant")
    mod.__file__ = oracle.__file__
    exec(compile(src, "oracle_mutant", "exec"), mod.__dict__)
    return mod


PY_PINS = {
    "sqrt_schur": P.test_sqrt_exact_matches_schur_sqrtm,
    "tridiag_dense": P.test_tridiagonal_root_matches_dense,
    "lanczos_full_dimension": P.test_lanczos_full_dimension_is_exact,
    "lanczos_eigenvector": P.test_lanczos_eigenvector_converges_in_one_step,
    "lanczos_tolerance": P.test_lanczos_tolerance_controls_error,
    "philox_kat": P.test_philox_known_answer_vectors,
    "soft_gradient": lambda o: IP.test_soft_repulsion_is_minus_energy_gradient(),
    "ab_euler_second_order": lambda o: IP.test_ab_step_first_step_is_euler_and_second_order(),
}


def _py_pins(monkeypatch, mod):
    monkeypatch.setattr(IP, "oracle", mod)
    held = {}
    for name, pin in PY_PINS.items():
        try:
            pin(mod)
            held[name] = True
        except AssertionError:
            held[name] = False
    return held


def test_unchanged_python_copy_passes_every_pin(monkeypatch):
    held = _py_pins(monkeypatch, _py_mutant())
    assert all(held.values()), held


PY_MUTATIONS = [
    ("tridiagonal_root_without_sqrt", "return Q @ (np.sqrt(lam) * Q[0, :])", "return Q @ (lam * Q[0, :])",
     {"tridiag_dense", "lanczos_full_dimension"}),
    ("lanczos_without_norm_of_W", "z = normW * tridiag_sqrt_e1(alpha, beta)", "z = tridiag_sqrt_e1(alpha, beta)",
     {"lanczos_full_dimension", "lanczos_eigenvector"}),
    ("square_root_transposed_operand", "return Q @ (root * (Q.T @ W))", "return Q.T @ (root * (Q @ W))",
     {"sqrt_schur"}),
    ("philox_weyl_constant", "_PHILOX_W1 = 0xBB67AE85", "_PHILOX_W1 = 0xBB67AE86", {"philox_kat"}),
    ("philox_round_word_order", "c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0",
     "c0, c1, c2, c3 = (hi0 ^ c1 ^ k0), lo1, (hi1 ^ c3 ^ k1), lo0", {"philox_kat"}),
    ("philox_key_schedule", "if rnd < 9:", "if rnd < 8:", {"philox_kat"}),
    ("soft_force_without_1_over_b", "U0 / b * np.exp((d_pair - r[m]) / b)", "U0 * np.exp((d_pair - r[m]) / b)",
     {"soft_gradient"}),
    ("adams_bashforth_history_sign", "1.5 * u - 0.5 * np.asarray(prev_u)", "1.5 * u + 0.5 * np.asarray(prev_u)",
     {"ab_euler_second_order"}),
]


@pytest.mark.parametrize("name,old,new,caught_by", PY_MUTATIONS, ids=[m[0] for m in PY_MUTATIONS])
def test_planted_python_mistake_fails_its_pins(monkeypatch, name, old, new, caught_by):
    held = _py_pins(monkeypatch, _py_mutant(old, new))
    failed = {k for k, ok in held.items() if not ok}
    assert caught_by <= failed, (name, held)
