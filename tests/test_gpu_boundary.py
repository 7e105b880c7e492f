"""Boundary conventions: APIC_CHECK input validation and the caller's
device allocator (apic_set_allocator).

APIC_CHECK must refuse non-finite v, C or normals and normals of neither
zero nor unit length, and otherwise change nothing (same bits, in the
deterministic mode).  A context whose scratch comes from the caller's
allocator must give the same bits as one using cudaMalloc, hand back every
block it took, and refuse an allocator set too late or a misaligned block.
"""
import numpy as np
import pytest

from paper_2108_02259_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def apic():
    import torch  # noqa: F401

    from paper_2108_02259_gb300 import apic as a, build

    build.build()
    return a


def _dev(s):
    import torch

    f = s.astype(np.float32)
    d = torch.device("cuda:0")

    def t(a, ty):
        return torch.as_tensor(np.ascontiguousarray(a), device=d, dtype=ty)

    return [t(f.x, torch.float64), t(f.v, torch.float32), t(f.C, torch.float32), t(f.m, torch.float32),
            t(f.nrm, torch.float32), t(f.body, torch.int32)]


def _step(apic, ctx, s, dev, flags):
    import torch

    r = apic.contact_step(ctx, *dev, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies, flags=flags)
    torch.cuda.synchronize()
    return r.v.clone(), r.C.clone()


def test_check_accepts_valid_input_unchanged(apic):
    import torch

    det, chk = apic.APIC_DETERMINISTIC, apic.APIC_CHECK
    s = scenes.four_bodies(scale=0.05)
    dev = _dev(s)
    with apic.Context(0) as ctx:
        a = _step(apic, ctx, s, dev, det)
        b = _step(apic, ctx, s, dev, det | chk)
        for _ in range(2):  # captured and replayed with the check
            c = _step(apic, ctx, s, dev, det | chk)
    assert all(torch.equal(p, q) for p, q in zip(a, b))
    assert all(torch.equal(p, q) for p, q in zip(a, c))


@pytest.mark.parametrize("what", ["v_nan", "C_inf", "nrm_nan", "nrm_not_unit"])
def test_check_rejects_bad_input(apic, what):
    import torch

    s = scenes.random_cloud(2000, n_bodies=2, seed=51, h=0.05, n_iter=2)
    X, V, Cc, M, NR, B = _dev(s)
    if what == "v_nan":
        V[5, 0] = float("nan")
        msg = "not finite"
    elif what == "C_inf":
        Cc[7, 1, 2] = float("inf")
        msg = "not finite"
    elif what == "nrm_nan":
        NR[3, 2] = float("nan")
        msg = "not finite"
    else:
        NR[11] = torch.tensor([0.5, 0.0, 0.0])
        msg = "unit length"
    with apic.Context(0) as ctx:
        # without the check the call goes through
        apic.contact_step(ctx, X, V, Cc, M, NR, B, s.h, s.mu, s.n_iter, n_bodies=2)
        with pytest.raises(apic.ApicError, match=msg):
            apic.contact_step(ctx, X, V, Cc, M, NR, B, s.h, s.mu, s.n_iter, n_bodies=2, flags=apic.APIC_CHECK)


def test_check_on_page_locked_host_arrays(apic):
    """With APIC_CHECK the host path stages every array before the cell
    kernel (no overlapped second copy) and still matches the device path."""
    import torch

    det, chk = apic.APIC_DETERMINISTIC, apic.APIC_CHECK
    s = scenes.four_bodies(scale=0.05, n_iter=3)
    f = s.astype(np.float32)

    def pinned(a, dt):
        a = np.ascontiguousarray(a, dt)
        t = torch.empty(a.shape, dtype=getattr(torch, np.dtype(dt).name)).pin_memory()
        t.numpy()[...] = a
        return t.numpy()

    hx = [pinned(f.x, np.float64), pinned(f.v, np.float32), pinned(f.C, np.float32), pinned(f.m, np.float32),
          pinned(f.nrm, np.float32), pinned(f.body, np.int32)]
    vo, Co = pinned(np.zeros_like(f.v), np.float32), pinned(np.zeros_like(f.C), np.float32)
    with apic.Context(0) as ctx:
        ref = _step(apic, ctx, s, _dev(s), det)
        for flags in (det | chk, det):
            apic.contact_step(ctx, *hx, s.h, s.mu, s.n_iter, n_bodies=s.n_bodies, flags=flags, v_out=vo, C_out=Co)
            assert np.array_equal(vo, ref[0].cpu().numpy()) and np.array_equal(Co, ref[1].cpu().numpy())


class _Counting:
    """torch's caching allocator behind counters."""

    def __init__(self, misalign=False):
        self.live, self.allocs, self.frees, self.misalign = {}, 0, 0, misalign

    def alloc(self, nbytes, device):
        import torch

        p = torch.cuda.caching_allocator_alloc(nbytes + (256 if self.misalign else 0), device)
        self.allocs += 1
        q = p + 16 if self.misalign else p
        self.live[q] = p
        return q

    def free(self, ptr, nbytes, device):
        import torch

        torch.cuda.caching_allocator_delete(self.live.pop(ptr))
        self.frees += 1


def test_caller_allocator_serves_all_scratch(apic):
    import torch

    det = apic.APIC_DETERMINISTIC
    s = scenes.four_bodies(scale=0.05)
    big = scenes.four_bodies(scale=0.2)  # a larger scene later makes buffers grow
    dev, dev_big = _dev(s), _dev(big)
    with apic.Context(0) as ref_ctx:
        ref = _step(apic, ref_ctx, s, dev, det)
        ref_big = _step(apic, ref_ctx, big, dev_big, det)
    cnt = _Counting()
    ctx = apic.Context(0)
    ctx.set_allocator(cnt.alloc, cnt.free)
    for _ in range(3):
        got = _step(apic, ctx, s, dev, det)
        assert all(torch.equal(p, q) for p, q in zip(got, ref))
    n0 = cnt.allocs
    got_big = _step(apic, ctx, big, dev_big, det)
    assert all(torch.equal(p, q) for p, q in zip(got_big, ref_big))
    assert n0 > 0 and cnt.allocs > n0 and cnt.frees > 0  # grew through the allocator
    got = _step(apic, ctx, s, dev, det)
    assert all(torch.equal(p, q) for p, q in zip(got, ref))
    with pytest.raises(apic.ApicError, match="set the allocator first"):
        ctx.set_allocator(cnt.alloc, cnt.free)
    ctx.close()
    assert cnt.frees == cnt.allocs and not cnt.live


def test_misaligned_allocator_is_refused(apic):
    s = scenes.random_cloud(1000, n_bodies=2, seed=53, h=0.05, n_iter=1)
    cnt = _Counting(misalign=True)
    ctx = apic.Context(0)
    ctx.set_allocator(cnt.alloc, cnt.free)
    with pytest.raises(apic.ApicError, match="aligned"):
        apic.contact_step(ctx, *_dev(s), s.h, s.mu, s.n_iter, n_bodies=2)
    ctx.close()
    assert cnt.frees == cnt.allocs and not cnt.live
