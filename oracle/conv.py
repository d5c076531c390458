"""Oracle: circular convolution / correlation on C^b, two independent engines.

Definitions (App. F; vectors 0-indexed):
    (a * c)[t]      = sum_{(i + j) mod b = t} a_i c_j                       (convolution)
    corr(x, y)[s]   = sum_d x[(d + s) mod b] conj(y[d])                      (correlation)
    <x, y>          = sum_t x_t conj(y_t)                                    (inner product)

Prop. 1 rests on corr(x, y) = F^{-1}(F(x) o conj(F(y))) and a * c = F^{-1}(F(a) o F(c)),
with F the unnormalised DFT F(x)_f = sum_t x_t exp(-2 pi i f t / b) and F^{-1} carrying 1/b.
The "direct" engine evaluates the sums over the nonzeros of the sparse argument; the "fft"
engine uses numpy's FFT as a library step.  Tests pin one against the other.

TEST INFRASTRUCTURE ONLY -- imported by tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline legs; the product path never calls it.
"""
from __future__ import annotations

import numpy as np


def inner(x: np.ndarray, y: np.ndarray) -> complex:
    """<x, y> = sum_t x_t conj(y_t)."""
    return complex(np.sum(np.asarray(x) * np.conj(np.asarray(y))))


def conv_direct(a: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Circular convolution by its definition, looping over the nonzeros of the sparser input."""
    a = np.asarray(a, dtype=np.complex128)
    c = np.asarray(c, dtype=np.complex128)
    if np.count_nonzero(a) > np.count_nonzero(c):
        a, c = c, a
    out = np.zeros_like(c)
    for i in np.nonzero(a)[0]:
        out += a[i] * np.roll(c, i)        # c shifted so that out[t] gets c[(t - i) mod b]
    return out


def corr_direct(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """corr(x, y)[s] = sum_d x[(d + s) mod b] conj(y[d]), looping over the nonzeros of y."""
    x = np.asarray(x, dtype=np.complex128)
    y = np.asarray(y, dtype=np.complex128)
    out = np.zeros_like(x)
    for d in np.nonzero(y)[0]:
        out += np.conj(y[d]) * np.roll(x, -d)    # entry s is x[(s + d) mod b]
    return out


def fft(x: np.ndarray) -> np.ndarray:
    """Unnormalised forward DFT, exp(-2 pi i f t / b)."""
    return np.fft.fft(np.asarray(x, dtype=np.complex128))


def ifft(X: np.ndarray) -> np.ndarray:
    """Inverse DFT carrying the 1/b factor."""
    return np.fft.ifft(np.asarray(X, dtype=np.complex128))


def conv_fft(a: np.ndarray, c: np.ndarray) -> np.ndarray:
    return ifft(fft(a) * fft(c))


def corr_fft(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """F^{-1}(F(x) o conj(F(y))) -- the left operand of the inner product in Prop. 1."""
    return ifft(fft(x) * np.conj(fft(y)))
