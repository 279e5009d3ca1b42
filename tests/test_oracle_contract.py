"""Pins of the contraction oracle (Sec. 5, Eqs. tmr, C_stoch2, timetrans)
against facts outside it: the trace identity of the one-end trick on a dense
inverse, a closed form for the identity propagator, time-reflection symmetry
and translation invariance of the free-field correlator."""
import numpy as np
import pytest

import synthetic
from oracle import contract as K
from oracle import dirac as D


def _dense_S(L, U, kappa, csw):
    return np.linalg.inv(D.dense_dirac(U, kappa, csw))


def _estimator_over_point_sources(S, L, y0):
    """The estimator of Eq. C_stoch2 summed over the 12 spin-colour point
    sources at every site of slice y0 (exact dilution of the slice)."""
    V = int(np.prod(L))
    slice_ = V // L[0]
    acc = np.zeros(L[0], dtype=np.complex128)
    for s in range(slice_):
        y = y0 * slice_ + s
        for e in range(12):
            eta = np.zeros(V * 12, dtype=np.complex128)
            eta[y * 12 + e] = 1.0
            b = (S @ eta).reshape(tuple(L) + (4, 3))
            # gamma_k is Hermitian: gamma5 gamma_k^dag eta = gamma5 gamma_k eta
            a = np.stack([(S @ K.spin_apply(K.gamma5_gamma(k), eta.reshape(tuple(L) + (4, 3))).reshape(-1))
                          .reshape(tuple(L) + (4, 3)) for k in (1, 2, 3)])
            acc += K.slice_correlator(a, b)
    return acc


def test_identity_propagator_closed_form():
    """S = 1: tr{gamma_k gamma_k} = 12 per site and k, so C(x0, y0) = -12 delta."""
    L = (4, 2, 2, 2)
    V = int(np.prod(L))
    C = K.correlator_from_propagator(np.eye(V * 12), L, 2)
    want = np.zeros(L[0])
    want[2] = -12.0
    assert np.abs(C - want).max() < 1e-14
    assert np.abs(_estimator_over_point_sources(np.eye(V * 12), L, 2) - want).max() < 1e-14


@pytest.mark.parametrize("y0", [0, 3])
def test_one_end_trick_equals_trace_formula(y0):
    """Summed over exact point sources of the slice, the estimator equals the
    trace formula of Eq. tmr (gamma5-hermiticity of S) on a random field."""
    L = (4, 2, 2, 2)
    U = synthetic.gauge_links(L, 0.4, 5)
    S = _dense_S(L, U, 0.125, 1.3)
    C = K.correlator_from_propagator(S, L, y0)
    assert np.abs(_estimator_over_point_sources(S, L, y0) - C).max() < 1e-13 * np.abs(C).max()
    assert np.abs(C.imag).max() < 1e-12 * np.abs(C).max()  # C is real (gamma5-hermiticity)


def test_free_field_reflection_and_translation():
    """Unit links: C(x0, y0) depends only on x0 - y0 and is symmetric under
    t -> L0 - t; the translation average of Eq. timetrans then equals C(t, 0)."""
    L = (6, 2, 2, 2)
    S = _dense_S(L, synthetic.free_links(L), 0.12, 1.0)
    Cm = np.stack([K.correlator_from_propagator(S, L, y0) for y0 in range(L[0])], axis=1)  # [x0, y0]
    for y0 in range(L[0]):
        assert np.abs(np.roll(Cm[:, y0], -y0) - Cm[:, 0]).max() < 1e-13
    c = Cm[:, 0]
    for t in range(1, L[0]):
        assert abs(c[t] - c[L[0] - t]) < 1e-13
    assert np.abs(K.translation_average(Cm) - c).max() < 1e-13
    assert np.all(c.real < 0)  # the sign Eq. tmr gives in the chiral basis


def test_correlator_gauge_invariant():
    """C(x0, y0) of Eq. tmr is a colour trace of gauge-covariant propagators:
    a random gauge transformation of the links leaves it unchanged (a dropped
    or misplaced colour index in the trace would not be invariant)."""
    L = (4, 2, 2, 2)
    U = synthetic.gauge_links(L, 0.4, 21)
    g = synthetic.random_su3(L, 1.0, 22)
    Ug = D.gauge_transform_links(U, g)
    for y0 in (0, 2):
        C = K.correlator_from_propagator(_dense_S(L, U, 0.125, 1.3), L, y0)
        Cg = K.correlator_from_propagator(_dense_S(L, Ug, 0.125, 1.3), L, y0)
        assert np.abs(Cg - C).max() < 1e-12 * np.abs(C).max()
