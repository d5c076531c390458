"""Step-wise parity of Alg. 1 between the CUDA path and the oracle.

Alg. 1 iterates a map (power update, median, normalisation) whose Jacobian can exceed 1 when the
sketch noise is comparable to the signal, so FP32 and FP64 runs started from the same inputs
separate after enough iterations, as two FP64 runs with different summation orders would.  The
comparison is therefore made one step at a time: every GPU iterate u_{t+1} is checked against
the oracle's power update applied to the GPU's own u_t, every eigenvalue estimate against the
oracle's T^(u,u,u) at the GPU's final iterate, the selection against the first argmax, and the
deflated sketches against the oracle's deflation with the GPU's (lambda^, u^) chained from the
input sketch.
"""
import numpy as np

import oracle as O


def normalise_rows(U):
    return U / np.linalg.norm(U, axis=-1, keepdims=True)


def check_rtpm_stepwise(res, S0, h, g, b, U0, T_it, rounds=None, steps=None, taus=None,
                        tol_vec=1e-4, tol_lam=1e-4):
    """res: robust_power_method(..., return_deflated=True, return_trace=True) on the host
    (numpy arrays); S0: [B][b] input sketches (complex128); h, g: [B][n]; U0: [k][L][n]."""
    lam = res["lam"]
    V = res["V"]
    tau = res["tau"]
    lam_all = res["lam_all"]
    U_it = res["U_iters"].astype(np.float64)
    k, L, n = U0.shape
    rounds = range(k) if rounds is None else rounds
    steps = range(T_it) if steps is None else steps
    taus = range(L) if taus is None else taus
    S = np.array(S0, dtype=np.complex128)
    checked = 0
    for r in range(k):
        if r in rounds:
            for t in steps:
                prev = normalise_rows(U0[r]) if t == 0 else U_it[r, t - 1]
                for tu in taus:
                    want, _ = O.power_step_sketched(S, prev[tu], h, g, b, "fft")
                    got = U_it[r, t, tu]
                    assert np.linalg.norm(got - want) <= tol_vec, (r, t, tu, np.linalg.norm(got - want))
                    checked += 1
            want_lam = np.array([O.eigenvalue_sketched(S, U_it[r, T_it - 1, tu], h, g, b, "fft")[0]
                                 for tu in range(L)])
            scale = max(1.0, np.max(np.abs(want_lam)))
            assert np.max(np.abs(lam_all[r] - want_lam)) <= tol_lam * scale, (r, lam_all[r], want_lam)
            # the GPU's choice is an argmax of the oracle's estimates within the tolerance
            assert want_lam[tau[r]] >= want_lam.max() - 2 * tol_lam * scale
        # the GPU reports the component it selected: a maximum of the round's eigenvalues, taken
        # in FP64 (the float trace is the FP64 median rounded to float)
        assert lam_all[r, tau[r]] == lam_all[r].max()
        assert np.float32(lam[r]) == lam_all[r, tau[r]]
        np.testing.assert_array_equal(V[r], U_it[r, T_it - 1, tau[r]].astype(np.float32))
        S = O.deflate_sketches(S, float(lam[r]), V[r].astype(np.float64), h, g, b, "fft")
    Sd = res["S_deflated"]
    err = np.linalg.norm(Sd - S) / np.linalg.norm(S)
    assert err <= tol_vec, err
    return checked


def check_rtpm_p_stepwise(res, S0, h, g, b, p, U0, T_it, tol_vec=1e-4, tol_lam=1e-4):
    """check_rtpm_stepwise for Alg. 1 of order p (oracle.orderp): every GPU iterate against the
    oracle's order-p power update of the GPU's previous iterate, every eigenvalue estimate, the
    first-argmax selection and the chained deflation.  h, g: [B][n]."""
    P = O.orderp
    lam, V, tau = res["lam"], res["V"], res["tau"]
    lam_all = res["lam_all"]
    U_it = res["U_iters"].astype(np.float64)
    k, L, n = U0.shape
    S = np.array(S0, dtype=np.complex128)
    checked = 0
    for r in range(k):
        for t in range(T_it):
            prev = normalise_rows(U0[r]) if t == 0 else U_it[r, t - 1]
            for tu in range(L):
                want, _ = P.power_step_p(S, prev[tu], h, g, b, p)
                got = U_it[r, t, tu]
                assert np.linalg.norm(got - want) <= tol_vec, (r, t, tu, np.linalg.norm(got - want))
                checked += 1
        want_lam = np.array([P.eigenvalue_p(S, U_it[r, T_it - 1, tu], h, g, b, p)[0] for tu in range(L)])
        scale = max(1.0, np.max(np.abs(want_lam)))
        assert np.max(np.abs(lam_all[r] - want_lam)) <= tol_lam * scale, (r, lam_all[r], want_lam)
        assert want_lam[tau[r]] >= want_lam.max() - 2 * tol_lam * scale
        assert tau[r] == int(np.argmax(lam_all[r]))
        assert lam[r] == np.float32(lam_all[r, tau[r]])
        np.testing.assert_array_equal(V[r], U_it[r, T_it - 1, tau[r]].astype(np.float32))
        S = P.deflate_p(S, float(lam[r]), V[r].astype(np.float64), h, g, b, p)
    err = np.linalg.norm(res["S_deflated"] - S) / np.linalg.norm(S)
    assert err <= tol_vec, err
    return checked
