"""The margins of the pivot search's FP32 filters, checked on the host.

The pivot-search kernels try each threshold test (Listing 1's 1x1 test, and
the 2x2 test's cancellation guard and growth bound, eq. (2.2)) first in FP32
on the magnitudes' bit patterns (truncated to 23 mantissa bits) with margins
of 2^-16, and skip the FP64 test only when FP32 proves its outcome.  This file
restates both the FP32 filters and the FP64 tests they stand in front of in
numpy (IEEE binary32 and binary64 arithmetic, round to nearest) and checks, on
inputs placed at relative distances from 1e-3 down to 1e-9 of each bound, that
a filter's verdict is never contradicted by the FP64 test.  It pins the error
analysis; the GPU tests check that the kernels' decisions equal the oracle's.
"""
import numpy as np

F32 = np.float32
M16 = F32(2.0 ** -16)


def key_f32(x):
    """Truncated binary32 value of |x| and whether |x| is 0 or within 2^+-32."""
    k = np.abs(np.asarray(x, np.float64)).view(np.uint64)
    e = (k >> np.uint64(52)).astype(np.int64)
    ok = (k == 0) | ((e >= 1023 - 32) & (e <= 1023 + 32))
    bits = ((k >> np.uint64(29)) - np.uint64(896 << 23)).astype(np.uint32)
    f = np.where(k == 0, F32(0.0), bits.view(np.float32))
    return f.astype(np.float32), ok


def fp64_2x2(a_tt, a_tm, a_mm, vt, vm, u, small):
    """The FP64 2x2 test in the kernels' rounding (True = accept)."""
    amax = np.maximum(np.abs(a_tt), np.maximum(np.abs(a_tm), np.abs(a_mm)))
    ds = 1.0 / amax
    d1 = (a_tm * ds) * a_tm
    d0 = (a_mm * ds) * a_tt
    det = d0 - d1
    guard = np.maximum(np.maximum(np.abs(d0) * 0.5, np.abs(d1) * 0.5), small)
    ok_det = np.abs(det) > guard
    lim = np.abs(det) * (1.0 / u)
    gt = (np.abs(a_mm) * vt + np.abs(a_tm) * vm) * ds
    gm = (np.abs(a_tm) * vt + np.abs(a_tt) * vm) * ds
    tiny = np.maximum(vt, vm) < small
    return ok_det & (tiny | ((gt <= lim) & (gm <= lim)))


def f32_reject_2x2(a_tt, a_tm, a_mm, vt, vm, u, small):
    """The kernels' FP32 filter: True where it proves the 2x2 test fails."""
    ftt, o1 = key_f32(a_tt)
    ftm, o2 = key_f32(a_tm)
    fmm, o3 = key_f32(a_mm)
    amax = np.maximum(np.abs(a_tt), np.maximum(np.abs(a_tm), np.abs(a_mm)))
    fmax, o4 = key_f32(amax)
    ok = o1 & o2 & o3 & o4 & (amax > 0)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        ds = (F32(1.0) / fmax).astype(np.float32)
        p0 = ((fmm * ds).astype(np.float32) * ftt).astype(np.float32)
        p1 = ((ftm * ds).astype(np.float32) * ftm).astype(np.float32)
        neg0 = np.signbit(a_mm) != np.signbit(a_tt)
        adet = np.abs(np.where(neg0, -p0, p0) - p1).astype(np.float32)
        err = (M16 * ((p0 + p1).astype(np.float32) + adet).astype(np.float32)).astype(np.float32)
        glow = ((F32(0.5) * np.maximum(p0, p1)).astype(np.float32) * (F32(1.0) - M16)).astype(np.float32)
        rej_det = ok & ((adet + err).astype(np.float32) < glow)
        fvt, o5 = key_f32(vt)
        fvm, o6 = key_f32(vm)
        fru, o7 = key_f32(1.0 / u)
        grow_ok = ok & o5 & o6 & o7 & (fru <= F32(2.0 ** 20)) & ~(np.maximum(vt, vm) < small)
        up = (fru * (F32(1.0) + F32(2.0 ** -21))).astype(np.float32)
        lim_up = ((((adet + err).astype(np.float32)) * up).astype(np.float32) * (F32(1.0) + M16)).astype(np.float32)
        gt = ((((fmm * fvt).astype(np.float32) + (ftm * fvm).astype(np.float32)).astype(np.float32)) * ds).astype(np.float32)
        gm = ((((ftm * fvt).astype(np.float32) + (ftt * fvm).astype(np.float32)).astype(np.float32)) * ds).astype(np.float32)
        one_m = F32(1.0) - M16
        rej_grow = grow_ok & (((gt * one_m).astype(np.float32) > lim_up) | ((gm * one_m).astype(np.float32) > lim_up))
    return rej_det | rej_grow


def f32_1x1(amm, maxm1, u):
    """The kernels' FP32 1x1 filter: 1 accept, 0 reject, -1 undecided."""
    fmm, o1 = key_f32(amm)
    fmx, o2 = key_f32(maxm1)
    fu, o3 = key_f32(np.full_like(amm, u))
    ok = o1 & o2 & o3
    lim = (fu * fmx).astype(np.float32)
    rej = ok & ((fmm * (F32(1.0) + M16)).astype(np.float32) < (lim * (F32(1.0) - M16)).astype(np.float32))
    acc = ok & ((fmm * (F32(1.0) - M16)).astype(np.float32) > (lim * (F32(1.0) + M16)).astype(np.float32))
    return np.where(acc, 1, np.where(rej, 0, -1))


def _near(rng, base, n):
    """base * (1 + s delta), s = +-1, delta log-uniform in [1e-9, 1e-3]."""
    d = 10.0 ** rng.uniform(-9, -3, n)
    s = rng.choice([-1.0, 1.0], n)
    return base * (1.0 + s * d)


def test_2x2_filter_never_contradicts_the_fp64_test():
    rng = np.random.default_rng(7)
    n = 400_000
    u, small = 0.01, 1e-20
    scale = 10.0 ** rng.uniform(-6, 6, n)
    a_tt = rng.standard_normal(n) * scale
    a_mm = rng.standard_normal(n) * scale
    # cancellation guard: a_tm^2 near a_tt a_mm / 2 (|det| = guard) or near 3/2 a_tt a_mm
    prod = np.abs(a_tt * a_mm)
    target = np.where(rng.random(n) < 0.5, 0.5, 1.5) * prod
    a_tm = np.sqrt(_near(rng, target, n)) * rng.choice([-1.0, 1.0], n)
    # growth bound: column maxima placing gt near lim
    amax = np.maximum(np.abs(a_tt), np.maximum(np.abs(a_tm), np.abs(a_mm)))
    det = np.abs(a_mm * a_tt - a_tm * a_tm) / amax
    w = rng.random(n)
    vt = w * det / u * amax / (np.abs(a_mm) + np.abs(a_tm) + 1e-300)
    vm = (1.0 - w) * det / u * amax / (np.abs(a_mm) + np.abs(a_tm) + 1e-300)
    vt, vm = _near(rng, vt, n), _near(rng, vm, n)
    # plus plain random cases
    a_tm[: n // 8] = rng.standard_normal(n // 8) * scale[: n // 8]
    vt[: n // 8] = np.abs(rng.standard_normal(n // 8)) * scale[: n // 8] * 30
    vm[: n // 8] = np.abs(rng.standard_normal(n // 8)) * scale[: n // 8] * 30
    exact = fp64_2x2(a_tt, a_tm, a_mm, vt, vm, u, small)
    rej = f32_reject_2x2(a_tt, a_tm, a_mm, vt, vm, u, small)
    assert not np.any(rej & exact), int(np.sum(rej & exact))
    # the filter settles most rejections, and leaves the close ones to FP64
    assert rej.sum() > 0.5 * (~exact).sum()


def test_1x1_filter_never_contradicts_the_fp64_test():
    rng = np.random.default_rng(11)
    n = 400_000
    u = 0.01
    maxm1 = np.abs(rng.standard_normal(n)) * 10.0 ** rng.uniform(-6, 6, n)
    amm = _near(rng, u * maxm1, n) * rng.choice([-1.0, 1.0], n)
    amm[: n // 8] = rng.standard_normal(n // 8) * maxm1[: n // 8]
    exact = np.abs(amm) >= u * maxm1
    f = f32_1x1(amm, maxm1, u)
    assert not np.any((f == 1) & ~exact)
    assert not np.any((f == 0) & exact)
    decided = f >= 0
    # cases more than 1e-4 from the bound, with both magnitudes within the
    # filter's range (2^+-32), are all decided in FP32
    far = np.abs(np.abs(amm) / (u * maxm1) - 1.0) > 1e-4
    in_range = key_f32(amm)[1] & key_f32(maxm1)[1]
    assert np.all(decided[far & in_range])
