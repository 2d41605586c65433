"""Comparison helpers of the GPU parity tests (imported by the test modules).

Every FP32 result is compared with the FP64 oracle twice:

* in the norm: relative L2 error <= 1e-5 (the target tolerance);
* element by element: |got - ref| <= 1e-4 * max|ref|, so that a single wrong
  vertex or task cannot hide inside a large norm.

A state that is advanced step by step (x_t, or the cotangent lam_t) is
dominated by its starting value, so the check is made on the increment
(x_T - x_0 against the oracle's) as well.  There the element bound adds the
rounding of storing the state in FP32 after every step: each store of a
value of size |x| can move it by half an ulp, at most 2^-24 |x|, so T steps
add up to T * 2^-24 * |x_T| per element on top of 1e-4 * max|increment|.
"""
import numpy as np

RTOL = 1e-5      # relative L2
ELEM = 1e-4      # element-wise, relative to the largest reference element
EPS32 = 2.0 ** -24


def _np(a):
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.asarray(a, np.float64)


def rel_l2(a, b):
    a, b = _np(a), _np(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def check_field(got, ref, name="", rtol=RTOL):
    """A quantity computed afresh (flux, SpMV output, weight gradient)."""
    got, ref = _np(got), _np(ref)
    assert got.shape == ref.shape, (name, got.shape, ref.shape)
    err = rel_l2(got, ref)
    assert err <= rtol, f"{name}: relative L2 error {err:.3e} > {rtol:g}"
    worst = float(np.max(np.abs(got - ref))) if got.size else 0.0
    bound = ELEM * float(np.max(np.abs(ref))) if ref.size else 0.0
    assert worst <= bound, f"{name}: max element error {worst:.3e} > {bound:.3e}"


def check_state(got, ref, base, steps, name="", rtol=RTOL):
    """A state advanced `steps` times from `base` (x0, or g for the adjoint)."""
    got, ref, base = _np(got), _np(ref), _np(base)
    err = rel_l2(got, ref)
    assert err <= rtol, f"{name}: relative L2 error {err:.3e} > {rtol:g}"
    dg, dr = got - base, ref - base
    if not np.any(dr):
        assert np.array_equal(got, ref), f"{name}: no increment expected"
        return
    inc = rel_l2(dg, dr)
    assert inc <= 10 * rtol + steps * EPS32 * np.linalg.norm(ref) / np.linalg.norm(dr), \
        f"{name}: increment relative L2 error {inc:.3e}"
    bound = ELEM * np.max(np.abs(dr)) + steps * EPS32 * np.abs(ref)
    excess = np.abs(dg - dr) - bound
    i = int(np.argmax(excess))
    assert excess.flat[i] <= 0, (f"{name}: element {i}: increment error {abs(dg - dr).flat[i]:.3e} "
                                 f"> bound {bound.flat[i]:.3e}")
