"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (written here, derived from the required accuracy of the FP32
form): v within 1e-5 of max|v|, C within 1e-4 of the C scale (max Frobenius
norm of the input or reference C, or 2 max|v| / h when both are zero),
momentum drift per step within 1e-6 of S_P = sum m|v| and
S_L = sum m (|x||v| + h^2 |C|_F).  The FP64 build must reach 1e-11.
"""
import numpy as np
import pytest

import discontinuity
import oracle
import parity_log
from paper_2108_02259_gb300 import scenes

pytestmark = pytest.mark.gpu

TOL_V32, TOL_C32, TOL_MOM32 = 1e-5, 1e-4, 1e-6
TOL64 = 1e-11


@pytest.fixture(scope="module")
def ctx():
    import torch  # noqa: F401

    from paper_2108_02259_gb300 import apic, build

    build.build()
    c = apic.Context(0)
    yield c
    c.close()


def run_gpu(ctx, s, dtype=np.float32, flags=0, mu_pair=None, stats=True, n_iter=None, mu=None, host=False):
    import torch

    from paper_2108_02259_gb300 import apic

    n_iter = s.n_iter if n_iter is None else n_iter
    mu = s.mu if mu is None else mu
    f = s.astype(dtype)
    if host:
        r = apic.contact_step(ctx, f.x, f.v, f.C, f.m, f.nrm, f.body, s.h, mu, n_iter, n_bodies=s.n_bodies,
                              mu_pair=mu_pair, flags=flags, stats=stats)
        return r.v.astype(np.float64), r.C.astype(np.float64), r.stats
    dev = torch.device("cuda:0")
    tdt = torch.float32 if dtype == np.float32 else torch.float64

    def t(a, dt):
        return torch.as_tensor(np.ascontiguousarray(a), device=dev, dtype=dt)

    r = apic.contact_step(ctx, t(f.x, torch.float64), t(f.v, tdt), t(f.C, tdt), t(f.m, tdt), t(f.nrm, tdt),
                          t(f.body, torch.int32), s.h, mu, n_iter, n_bodies=s.n_bodies, mu_pair=mu_pair,
                          flags=flags, stats=stats)
    torch.cuda.synchronize()
    return r.v.cpu().double().numpy(), r.C.cpu().double().numpy(), r.stats


def run_oracle(s, flags=0, mu_pair=None, n_iter=None, mu=None):
    n_iter = s.n_iter if n_iter is None else n_iter
    mu = s.mu if mu is None else mu
    return oracle.contact_step(s.x, s.v, s.C, s.m, s.nrm, s.body, s.h, mu, n_iter, n_bodies=s.n_bodies,
                               mu_pair=mu_pair, flags=flags)


def scales(s, ref_C):
    vs = max(np.abs(s.v).max(), 1e-300)
    cs = max(np.linalg.norm(s.C.reshape(-1, 9), axis=1).max(), np.linalg.norm(ref_C.reshape(-1, 9), axis=1).max())
    if cs == 0:
        cs = 2 * vs / s.h
    sP = np.sum(s.m * np.linalg.norm(s.v, axis=1))
    sL = np.sum(s.m * (np.linalg.norm(s.x, axis=1) * np.linalg.norm(s.v, axis=1)
                       + s.h * s.h * np.linalg.norm(s.C.reshape(-1, 9), axis=1)))
    return vs, cs, sP, sL


def check(s, got, ref, tol_v, tol_c, tol_mom=None, label="", count_multibody=True, env=None):
    """env = (v envelope, C envelope) from discontinuity.envelope: the errors
    are then measured beyond the oracle's own change at the step of the
    Sec. 2.3 rule, element by element."""
    v, Cm, st = got
    rv, rC, rst = ref
    vs, cs, sP, sL = scales(s, rC)
    if env is None:
        ev = np.abs(v - rv).max() / vs
        ec = np.abs(Cm - rC).max() / cs
    else:
        ev = discontinuity.excess(v, rv, env[0], vs)
        ec = discontinuity.excess(Cm, rC, env[1], cs)
    parity_log.record(label, s.n, {"v": ev, "C": ec}, {"v": tol_v, "C": tol_c})
    assert ev <= tol_v, f"{label} v error {ev:.3e} > {tol_v}"
    assert ec <= tol_c, f"{label} C error {ec:.3e} > {tol_c}"
    if tol_mom is not None and st is not None:
        assert np.abs(st["P_out"] - st["P_in"]).max() <= tol_mom * sP, f"{label} linear momentum drift"
        assert np.abs(st["L_out"] - st["L_in"]).max() <= tol_mom * sL, f"{label} angular momentum drift"
        # the device's own FP64 reduction of the input agrees with the oracle's
        assert np.abs(st["P_in"] - rst["P_in"]).max() <= 1e-6 * sP
        assert np.abs(st["L_in"] - rst["L_in"]).max() <= 1e-6 * sL
        if count_multibody:
            assert st["multibody_nodes"] == rst["multibody_nodes"], (st["multibody_nodes"], rst["multibody_nodes"])
    return ev, ec


# ------------------------------------------------------------ configs ----

def test_two_cubes_fp64(ctx):
    s = scenes.two_cubes(mu=0.3, n_iter=10)
    check(s, run_gpu(ctx, s, np.float64), run_oracle(s), TOL64, TOL64, 1e-12, "two cubes fp64")


def test_two_cubes_fp32(ctx):
    s = scenes.two_cubes(mu=0.3, n_iter=10)
    check(s, run_gpu(ctx, s, np.float32), run_oracle(s), TOL_V32, TOL_C32, TOL_MOM32, "two cubes fp32")


@pytest.mark.parametrize("mu,n_iter", [(0.0, 4), (0.3, 0), (2.0, 3)])
def test_two_cubes_variants(ctx, mu, n_iter):
    s = scenes.two_cubes(mu=mu, n_iter=n_iter)
    check(s, run_gpu(ctx, s), run_oracle(s), TOL_V32, TOL_C32, TOL_MOM32, f"two cubes mu={mu} N={n_iter}")


def test_four_bodies_small(ctx):
    """The 4-body scene at 1/20 size: several grid blocks, ragged items."""
    s = scenes.four_bodies(scale=0.05)
    check(s, run_gpu(ctx, s), run_oracle(s), TOL_V32, TOL_C32, TOL_MOM32, "four bodies small")


def test_four_bodies_full(ctx):
    """The full 200,000-node 4-body scene (h = 1/256, N = 8), every particle."""
    s = scenes.four_bodies()
    check(s, run_gpu(ctx, s), run_oracle(s), TOL_V32, TOL_C32, TOL_MOM32, "four bodies full")


def test_four_bodies_full_fp64(ctx):
    s = scenes.four_bodies()
    check(s, run_gpu(ctx, s, np.float64), run_oracle(s), TOL64, TOL64, 1e-12, "four bodies fp64")


@pytest.mark.parametrize("seed,nb,n_iter,origin", [(1, 2, 3, (0, 0, 0)), (2, 5, 2, (-3.3, 0.7, -0.05)),
                                                   (3, 32, 1, (10.0, -20.0, 5.0))])
def test_random_nonaffine(ctx, seed, nb, n_iter, origin):
    """Random non-affine states, dense clouds (many particles per cell),
    negative coordinates, up to 32 bodies."""
    s = scenes.random_cloud(3000, n_bodies=nb, seed=seed, h=0.1, n_iter=n_iter, origin=origin, spread=1.3)
    check(s, run_gpu(ctx, s), run_oracle(s), TOL_V32, TOL_C32, TOL_MOM32, f"random seed={seed}")
    check(s, run_gpu(ctx, s, np.float64), run_oracle(s), TOL64, TOL64, 1e-12, f"random fp64 seed={seed}")


def test_pic_and_sep23(ctx):
    from paper_2108_02259_gb300 import apic

    s = scenes.four_bodies(scale=0.02)
    check(s, run_gpu(ctx, s, flags=apic.APIC_VARIANT_PIC), run_oracle(s, flags=oracle.FLAG_PIC),
          TOL_V32, TOL_C32, None, "pic")
    # the Sec. 2.3 rule is a step at dn = 0 (tests/discontinuity.py): beyond the
    # oracle's own change under 1e-6 relative input changes
    ref = run_oracle(s, flags=oracle.FLAG_SEP23)
    _, _, env_v, env_C = discontinuity.envelope(
        lambda v, C: oracle.contact_step(s.x, v, C, s.m, s.nrm, s.body, s.h, s.mu, s.n_iter,
                                         n_bodies=s.n_bodies, flags=oracle.FLAG_SEP23)[:2], s.v, s.C)
    check(s, run_gpu(ctx, s, flags=apic.APIC_VARIANT_SEP23), ref, TOL_V32, TOL_C32, TOL_MOM32,
          "sep23 (beyond the oracle's envelope)", env=(env_v, env_C))


def test_mu_pair(ctx):
    s = scenes.random_cloud(2000, n_bodies=4, seed=9, h=0.12, n_iter=3)
    rng = np.random.default_rng(10)
    mp = rng.uniform(0.1, 0.5, (4, 4))
    mp = np.triu(mp) + np.triu(mp, 1).T
    check(s, run_gpu(ctx, s, mu_pair=mp), run_oracle(s, mu_pair=mp), TOL_V32, TOL_C32, TOL_MOM32, "mu_pair")
    check(s, run_gpu(ctx, s, np.float64, mu_pair=mp), run_oracle(s, mu_pair=mp), TOL64, TOL64, None, "mu_pair fp64")


def test_host_pointer_path(ctx):
    s = scenes.four_bodies(scale=0.02)
    a = run_gpu(ctx, s)
    b = run_gpu(ctx, s, host=True)
    check(s, b, run_oracle(s), TOL_V32, TOL_C32, TOL_MOM32, "host ptrs")
    vs = np.abs(s.v).max()
    assert np.abs(a[0] - b[0]).max() <= 2 * TOL_V32 * vs


# ------------------------------------------------------------ edges ----

def test_empty(ctx):
    s = scenes.random_cloud(1, seed=0)
    s0 = scenes.Scene(s.x[:0], s.v[:0], s.C[:0], s.m[:0], s.nrm[:0], s.body[:0], 1, 0.1, 0.3, 2)
    v, Cm, st = run_gpu(ctx, s0)
    assert v.shape == (0, 3) and Cm.shape == (0, 3, 3)


def test_single_particle_and_single_cell(ctx):
    for n in (1, 2, 40):
        s = scenes.random_cloud(n, n_bodies=2, seed=n, h=1.0, spread=0.999, origin=(5.0, 5.0, 5.0), n_iter=2)
        check(s, run_gpu(ctx, s), run_oracle(s), TOL_V32, TOL_C32, TOL_MOM32, f"n={n}")


def test_single_rigid_body_unchanged(ctx):
    s = scenes.four_bodies(scale=0.05)
    keep = s.body == 2
    s1 = scenes.Scene(s.x[keep], s.v[keep], s.C[keep], s.m[keep], s.nrm[keep], np.zeros(keep.sum(), np.int32),
                      1, s.h, 0.3, 8)
    v, Cm, st = run_gpu(ctx, s1)
    vs = np.abs(s1.v).max()
    assert np.abs(v - s1.v).max() <= TOL_V32 * vs
    assert np.abs(Cm - s1.C).max() <= TOL_C32 * np.abs(s1.C).max()
    assert st["multibody_nodes"] == 0


def test_cell_boundaries(ctx):
    """Particles exactly on grid lines (t = 0) and just below them."""
    rng = np.random.default_rng(77)
    h = 0.25
    base = rng.integers(-8, 8, (400, 3)).astype(np.float64) * h
    x = np.concatenate([base, base - 1e-9, base + 0.5 * h])
    n = x.shape[0]
    s = scenes.Scene(x, rng.standard_normal((n, 3)), rng.standard_normal((n, 3, 3)), rng.uniform(0.5, 1.5, n),
                     np.zeros((n, 3)), rng.integers(0, 3, n).astype(np.int32), 3, h, 0.3, 2)
    # The multi-body node count is not compared here: 1e-9 below a grid line
    # the offset t = 1 - 4e-9 rounds to 1 in FP32, so a node whose FP64 weight
    # is ~1e-17 receives no mass on the FP32 path and is not counted.
    check(s, run_gpu(ctx, s), run_oracle(s), TOL_V32, TOL_C32, TOL_MOM32, "cell boundaries",
          count_multibody=False)
    check(s, run_gpu(ctx, s, np.float64), run_oracle(s), TOL64, TOL64, 1e-12, "cell boundaries fp64")


def test_invalid_inputs_rejected(ctx):
    from paper_2108_02259_gb300 import apic

    s = scenes.random_cloud(50, n_bodies=2, seed=5)
    bad = s.astype(np.float32)
    bad.body[3] = 7
    with pytest.raises(apic.ApicError) as e:
        apic.contact_step(ctx, bad.x, bad.v, bad.C, bad.m, bad.nrm, bad.body, s.h, 0.3, 2, n_bodies=2)
    assert e.value.code == apic.APIC_ERR_INVALID_ARG
    bad = s.astype(np.float32)
    bad.m[0] = 0.0
    with pytest.raises(apic.ApicError):
        apic.contact_step(ctx, bad.x, bad.v, bad.C, bad.m, bad.nrm, bad.body, s.h, 0.3, 2)
    f = s.astype(np.float32)
    for h, mu, N in ((0.0, 0.3, 2), (0.1, -1.0, 2), (0.1, 0.3, -1), (np.inf, 0.3, 1)):
        with pytest.raises(apic.ApicError):
            apic.contact_step(ctx, f.x, f.v, f.C, f.m, f.nrm, f.body, h, mu, N)
    x = f.x.copy()
    x[1, 0] = np.nan
    with pytest.raises(apic.ApicError):
        apic.contact_step(ctx, x, f.v, f.C, f.m, f.nrm, f.body, s.h, 0.3, 2)
    # the context is still usable afterwards
    check(s, run_gpu(ctx, s), run_oracle(s), TOL_V32, TOL_C32, TOL_MOM32, "after errors")


def test_repeat_calls_reuse_scratch(ctx):
    s = scenes.four_bodies(scale=0.02)
    a = run_gpu(ctx, s)
    nbytes = ctx.scratch_bytes()
    b = run_gpu(ctx, s)
    assert ctx.scratch_bytes() == nbytes
    vs = np.abs(s.v).max()
    assert np.abs(a[0] - b[0]).max() <= 2 * TOL_V32 * vs


def test_page_table_box_reuse_and_refit(ctx):
    """The page-table box of one step is reused by the next when the
    particles still fit (a small shift) and refitted when they do not (a
    large shift); results match the oracle either way."""
    base = scenes.four_bodies(scale=0.02)
    for shift_cells in (0, 5, 3, 400, -7):
        s = scenes.Scene(base.x + shift_cells * base.h, base.v, base.C, base.m, base.nrm, base.body, base.n_bodies,
                         base.h, base.mu, 4)
        check(s, run_gpu(ctx, s), run_oracle(s), TOL_V32, TOL_C32, TOL_MOM32, f"shift {shift_cells} cells")


def _subset(s, keep, bodies):
    """The particles of `bodies` only, renumbered 0.. (for the oracle)."""
    remap = np.full(s.n_bodies, -1, np.int32)
    remap[list(bodies)] = np.arange(len(bodies), dtype=np.int32)
    mp = None if s.mu_pair is None else s.mu_pair[np.ix_(list(bodies), list(bodies))]
    return scenes.Scene(s.x[keep], s.v[keep], s.C[keep], s.m[keep], s.nrm[keep], remap[s.body[keep]], len(bodies),
                        s.h, s.mu, s.n_iter, mp)


def test_eight_bodies_full_size(ctx):
    """The 4,000,000-node 8-body scene (h = 1/512, per-pair mu, N = 8) as one
    launch, every particle against the oracle.  Its four approaching pairs
    (bodies 2k and 2k+1) are ~0.3 apart, far beyond the 2h stencil reach, so
    the oracle run on one pair alone gives exactly the full-scene answer for
    that pair's 1,000,000 particles; the four pairs run in parallel threads
    (the oracle holds no global state).  The full scene must also keep its
    momentum."""
    from concurrent.futures import ThreadPoolExecutor

    s = scenes.eight_bodies()
    v, Cm, st = run_gpu(ctx, s, mu_pair=s.mu_pair)
    vs, _, sP, sL = scales(s, s.C)
    assert np.abs(st["P_out"] - st["P_in"]).max() <= TOL_MOM32 * sP
    assert np.abs(st["L_out"] - st["L_in"]).max() <= TOL_MOM32 * sL
    pairs = []
    for k in range(4):
        keep = (s.body == 2 * k) | (s.body == 2 * k + 1)
        pairs.append((keep, _subset(s, keep, (2 * k, 2 * k + 1))))
    with ThreadPoolExecutor(4) as ex:
        refs = list(ex.map(lambda ks: run_oracle(ks[1], mu_pair=ks[1].mu_pair), pairs))
    for k, ((keep, sub), ref) in enumerate(zip(pairs, refs)):
        check(sub, (v[keep], Cm[keep], None), ref, TOL_V32, TOL_C32, None, f"eight bodies, pair {k} of full scene")


def test_limits_rejected_cleanly():
    """The documented limits fail with their error codes and leave the
    context usable: |x/h| >= 2^29, a page-table box beyond 2^28 blocks,
    more than 32 bodies, and a scene whose scratch exceeds the context's HBM
    budget."""
    from paper_2108_02259_gb300 import apic

    ok = scenes.random_cloud(200, n_bodies=2, seed=9, h=0.1, n_iter=2)
    with apic.Context(0, hbm_budget_bytes=8 << 20) as c:
        f = ok.astype(np.float32)
        far = f.x.copy()
        far[0] = [2.0 ** 29 * ok.h * 1.5, 0.0, 0.0]
        with pytest.raises(apic.ApicError) as e:
            apic.contact_step(c, far, f.v, f.C, f.m, f.nrm, f.body, ok.h, 0.3, 2, n_bodies=2)
        assert e.value.code == apic.APIC_ERR_INVALID_ARG and "position" in str(e.value)
        spread = f.x.copy()
        spread[0] = [1e4, 1e4, 1e4]  # a bounding box of ~10^15 grid blocks
        with pytest.raises(apic.ApicError) as e:
            apic.contact_step(c, spread, f.v, f.C, f.m, f.nrm, f.body, ok.h, 0.3, 2, n_bodies=2)
        assert e.value.code == apic.APIC_ERR_INVALID_ARG and "page-table" in str(e.value)
        with pytest.raises(apic.ApicError) as e:
            apic.contact_step(c, f.x, f.v, f.C, f.m, f.nrm, f.body, ok.h, 0.3, 2, n_bodies=33)
        assert e.value.code == apic.APIC_ERR_INVALID_ARG
        big = scenes.four_bodies(scale=0.2).astype(np.float32)  # 40,000 nodes: more scratch than 8 MiB
        with pytest.raises(apic.ApicError) as e:
            apic.contact_step(c, big.x, big.v, big.C, big.m, big.nrm, big.body, 1 / 256, 0.3, 2, n_bodies=4)
        assert e.value.code == apic.APIC_ERR_OUT_OF_MEMORY
        assert c.scratch_bytes() <= 8 << 20
        r = apic.contact_step(c, f.x, f.v, f.C, f.m, f.nrm, f.body, ok.h, ok.mu, ok.n_iter, n_bodies=2)
        ref = run_oracle(ok)
        check(ok, (r.v.astype(np.float64), r.C.astype(np.float64).reshape(-1, 3, 3), None), ref, TOL_V32,
              TOL_C32, None, "after limits", count_multibody=False)


@pytest.mark.parametrize("case", ["two_cubes_fp64", "four_bodies", "cloud", "affine_cloud"])
def test_energy_diagnostics(ctx, case):
    """apic_stats E_in / E_out: the generalised kinetic energy (1/2) sum m
    (|v|^2 + (h^2/2) |C|_F^2) of the inputs and outputs, in FP64 on the
    device.  Each matches the same sum over the arrays on the host, E_out
    matches the oracle's output energy, contact dissipates it, and an affine
    velocity field keeps it."""
    dt = np.float32
    if case == "two_cubes_fp64":
        s, dt = scenes.two_cubes(mu=0.3, n_iter=10), np.float64
    elif case == "four_bodies":
        s = scenes.four_bodies(scale=0.05)
    elif case == "cloud":
        s = scenes.random_cloud(3000, n_bodies=3, seed=5, h=0.05, n_iter=4)
    else:
        s = scenes.random_cloud(3000, n_bodies=3, seed=6, h=0.05, n_iter=4, affine=True)

    def energy(v, Cm):
        return 0.5 * np.sum(s.m.astype(dt).astype(np.float64) * (np.sum(v * v, axis=1)
                                                                 + 0.5 * s.h * s.h * np.sum(Cm.reshape(-1, 9) ** 2, axis=1)))

    v, Cm, st = run_gpu(ctx, s, dtype=dt)
    f = s.astype(dt)
    e_in_host = energy(f.v.astype(np.float64), f.C.astype(np.float64))
    assert abs(st["E_in"] - e_in_host) <= 1e-12 * e_in_host
    assert abs(st["E_out"] - energy(v, Cm)) <= 1e-12 * e_in_host
    rv, rC, _ = run_oracle(s)
    e_ref = energy(rv, rC)
    tol = 1e-12 if dt == np.float64 else 1e-5
    assert abs(st["E_out"] - e_ref) <= tol * e_in_host, (st["E_out"], e_ref)
    if case == "affine_cloud":
        assert abs(st["E_out"] - st["E_in"]) <= 10 * tol * st["E_in"]
    else:
        assert st["E_out"] < st["E_in"]
