"""The device-memory hook (lbm_allocator): forests, batches and nets take their device memory from
the caller's allocator; the Python binding routes it to torch's CUDA caching allocator."""
import ctypes

import numpy as np
import pytest

from paper_1508_07982_gb300 import inputs


def _refined_box(B, lmax=2):
    """Periodic 64^3 box with two nested refined boxes (three levels)."""
    regions = [("box", 1, (16, 16, 0), (48, 48, 64)), ("box", 2, (24, 24, 16), (40, 40, 48))][:lmax]
    return inputs.periodic_case(n=64, B=B, collision="trt", omega=1.7, regions=regions, lmax=lmax)


def _lbm_host():
    from paper_1508_07982_gb300 import build, lbm
    build.build()
    return lbm


def test_a_hook_with_alloc_but_no_release_is_rejected_before_any_cuda_call():
    lbm = _lbm_host()
    hook = lbm.Allocator(lbm.ALLOC_FN(lambda n, s, u: None), lbm.RELEASE_FN(), None)
    case = _refined_box(8)
    with pytest.raises(lbm.LBMError) as e:
        lbm.Forest(case, stream=0, allocator=hook)
    assert e.value.status == lbm.LBM_EINVAL and "release" in str(e.value)
    with pytest.raises(lbm.LBMError) as e:
        lbm.Net(stream=0, allocator=hook)
    assert e.value.status == lbm.LBM_EINVAL


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return _lbm_host()


def _pdf_bytes(lbm, case, esize):
    """Both PDF grids of every level: owned and ghost blocks, B^3 cells each."""
    p = lbm.Plan(case)
    blocks = [p.counts(L)["blocks"] + p.counts(L)["ghost_blocks"] for L in range(p.nlev)]
    return sum(2 * 19 * esize * n * case["B"] ** 3 for n in blocks)


class _Counting:
    """A hook over torch's caching allocator that records every call and can refuse the k-th
    allocation or hand out a pointer off the 256-byte grid."""

    def __init__(self, lbm, fail_at=None, offset=0):
        import torch
        self.torch, self.fail_at, self.offset = torch, fail_at, offset
        self.calls, self.live, self.released = 0, {}, []
        self.hook = lbm.Allocator(lbm.ALLOC_FN(self._alloc), lbm.RELEASE_FN(self._release), None)

    def _alloc(self, nbytes, stream, user):
        self.calls += 1
        if self.fail_at is not None and self.calls == self.fail_at:
            return None
        base = self.torch.cuda.caching_allocator_alloc(int(nbytes) + 256, stream=int(stream or 0))
        p = base + self.offset
        self.live[p] = (base, int(nbytes))
        return p

    def _release(self, ptr, nbytes, stream, user):
        base, n = self.live.pop(int(ptr))
        assert n == int(nbytes)
        self.released.append(n)
        self.torch.cuda.caching_allocator_delete(base)


@pytest.mark.gpu
@pytest.mark.parametrize("precision,esize", [("fp64", 8), ("fp32s", 4), ("fp16s", 2)])
def test_forest_memory_comes_from_torch_and_returns_to_it(lbm, precision, esize):
    import torch
    case = _refined_box(16)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    f = lbm.Forest(case, precision=precision)
    grown = torch.cuda.memory_allocated() - base
    need = _pdf_bytes(lbm, case, esize)
    # the rest (tables, staging, per-warp totals) is below 42 bytes per cell, less than the PDFs
    assert need <= grown <= 2 * need + 16 * 2**20, (grown, need)
    # the runtime's own cudaMalloc path does not touch torch's pool
    g = lbm.Forest(case, precision=precision, allocator=None)
    assert torch.cuda.memory_allocated() - base == grown
    field = inputs.taylor_green_field(64)
    for h in (f, g):
        h.init_fields(field)
        h.step_coarse(3)
    for L in range(f.nlev):
        a, b = f.get_pdfs(L), g.get_pdfs(L)
        assert np.array_equal(np.isnan(a), np.isnan(b))
        assert np.array_equal(a[~np.isnan(a)], b[~np.isnan(b)])
    # lazily allocated buffers (residual history, autotuning snapshot) go through the hook too
    f.velocity_residual()
    f.velocity_residual()
    f.autotune(2)
    f.close()
    g.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base


@pytest.mark.gpu
def test_every_allocation_and_release_passes_through_the_hook(lbm):
    case = _refined_box(8)
    h = _Counting(lbm)
    f = lbm.Forest(case, precision="fp32s", allocator=h.hook)
    f.init_fields(inputs.uniform_field())
    f.step_coarse(2)
    f.velocity_residual()
    b = lbm.Batch([f], allocator=h.hook)
    b.step(2)
    assert h.calls > 20 and len(h.live) == h.calls
    b.close()
    f.close()
    assert h.live == {} and len(h.released) == h.calls


@pytest.mark.gpu
@pytest.mark.parametrize("fail_at", [1, 7, 25])
def test_a_refused_allocation_gives_enomem_and_frees_what_was_taken(lbm, fail_at):
    case = _refined_box(8)
    h = _Counting(lbm, fail_at=fail_at)
    with pytest.raises(lbm.LBMError) as e:
        lbm.Forest(case, precision="fp64", allocator=h.hook)
    assert e.value.status == lbm.LBM_ENOMEM
    assert h.live == {}


@pytest.mark.gpu
def test_a_pointer_off_the_256_byte_grid_is_handed_back_and_refused(lbm):
    case = _refined_box(8, lmax=1)
    h = _Counting(lbm, offset=16)
    with pytest.raises(lbm.LBMError) as e:
        lbm.Forest(case, precision="fp32s", allocator=h.hook)
    assert e.value.status == lbm.LBM_ENOMEM
    assert h.live == {} and h.calls == 1


@pytest.mark.gpu
def test_net_memory_comes_from_torch(lbm):
    import torch
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    net = lbm.Net(layers=3, in_channels=6, out_channels=4)
    params = torch.cuda.memory_allocated() - base
    assert params >= 4 * 4 * net.num_params()          # parameters, gradients, two Adam moments
    x = torch.zeros((2, 12, 12, 12, 16), dtype=torch.bfloat16, device="cuda")
    net.forward(x)
    acts = 5 * 2 * 12 ** 3 * 16 * 2                      # 3 layers + 1 output + 2 gradient buffers, at least
    assert torch.cuda.memory_allocated() - base - params - x.numel() * 2 >= acts
    net.close()
    del x
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base
