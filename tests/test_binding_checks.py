"""The binding checks caller-supplied tensors (sizes, shapes, devices) before
any library call: the C entry points receive only pointers, so a buffer of
the wrong size would otherwise be read or written out of bounds on the GPU.
Runs on the CPU: the library is replaced by a stub that fails if called, and
the CUDA-tensor requirement is relaxed to CPU tensors; correctly sized
arguments must get through to the stub."""
import numpy as np
import pytest
import torch

import paper_2404_16039_gb300 as vla

F32, F64, I32 = torch.float32, torch.float64, torch.int32


class _LibraryReached(Exception):
    pass


class _NoLib:
    def __getattr__(self, name):
        raise _LibraryReached(name)


@pytest.fixture
def b(monkeypatch):
    def lenient(t, dtype=None):
        if not isinstance(t, torch.Tensor):
            raise TypeError("expected a tensor")
        if not t.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        if dtype is not None and t.dtype != dtype:
            raise TypeError(f"expected {dtype}")
        return t

    monkeypatch.setattr(vla, "_req", lenient)
    monkeypatch.setattr(vla, "lib", lambda: _NoLib())
    monkeypatch.setattr(vla, "_stream", lambda stream=None: None)
    monkeypatch.setattr(vla, "quad_rule", lambda sdim, gqo: (np.zeros((4, sdim + 1)), np.full(4, 0.25)))
    return vla


def _mesh(dim=3, order=1, nn=5, ne=2, nfb=4, nnz=13):
    m = object.__new__(vla.Mesh)
    m.__dict__.update(dim=dim, order=order, nlb=vla._nlb(dim, order), nn=nn, ne=ne, nfb=nfb, nnz=nnz,
                      device=torch.device("cpu"), _h=None)
    return m


def test_page_outputs_must_have_the_result_size(b):
    A, B = torch.zeros((4, 3, 3)), torch.zeros((4, 3, 3))
    with pytest.raises(ValueError):
        b.amtam(A, B, out=torch.zeros((4, 3, 2)))
    with pytest.raises(ValueError):
        b.amdet(A, out=torch.zeros(3))
    with pytest.raises(ValueError):
        b.aminv(A, det=torch.zeros(5))
    with pytest.raises(ValueError):
        b.avtam(torch.zeros((4, 3)), A, out=torch.zeros((4, 2)))
    with pytest.raises(ValueError):
        b.amsv(A, torch.zeros(3), out=torch.zeros((4, 2)))
    with pytest.raises(ValueError):
        b.avtamav(torch.zeros((4, 3)), A, torch.zeros((4, 2)))
    with pytest.raises(ValueError):
        b.avtamav(torch.zeros((4, 3)), torch.zeros((4, 2, 3)), torch.zeros((4, 3)))
    with pytest.raises(_LibraryReached):        # the right sizes get through
        b.amtam(A, B, out=torch.zeros((4, 3, 3)))
    with pytest.raises(_LibraryReached):
        b.avtamav(torch.zeros((4, 3)), A, torch.zeros((4, 3)), out=torch.zeros(4))


def test_mesh_arrays_must_match_the_element_order(b):
    coords = torch.zeros((5, 3), dtype=F64)
    with pytest.raises(ValueError):
        b.Mesh(coords, torch.zeros((2, 4), dtype=I32), order=2)            # P2 tets have 10 nodes
    with pytest.raises(ValueError):
        b.Mesh(coords, torch.zeros((2, 4), dtype=I32), faces=torch.zeros((4, 2), dtype=I32))
    with pytest.raises(ValueError):
        b.element_pages_static(coords, torch.zeros((2, 3), dtype=I32))
    # the allocation-free path reads its indices as given: the binding checks them first
    for bad in (5, -1):
        el = torch.zeros((2, 4), dtype=I32)
        el[1, 2] = bad
        with pytest.raises(vla.VlaError) as ei:
            b.element_pages_static(coords, el)
        assert ei.value.status == vla.VLA_ERR_INDEX_OOB
    with pytest.raises(_LibraryReached):
        b.element_pages_static(coords, torch.tensor([[0, 1, 2, 4], [1, 2, 3, 4]], dtype=I32))
    with pytest.raises(ValueError):
        b.autotune(torch.zeros((5, 2), dtype=F64), torch.zeros((2, 4), dtype=I32))
    with pytest.raises(_LibraryReached):
        b.Mesh(coords, torch.zeros((2, 4), dtype=I32), faces=torch.zeros((4, 3), dtype=I32))


def test_mesh_buffers_must_have_the_mesh_sizes(b):
    m = _mesh()
    with pytest.raises(ValueError):
        m.assemble(K=torch.zeros(12, dtype=F64))
    with pytest.raises(ValueError):
        m.assemble(vol=torch.zeros(3, dtype=F64))
    with pytest.raises(ValueError):
        m.boundary(normals=torch.zeros((4, 2), dtype=F64))
    with pytest.raises(ValueError):
        m.rhs(2, torch.zeros((2, 3), dtype=F64))                           # 4 points per element
    with pytest.raises(ValueError):
        m.rhs(2, torch.zeros((2, 4), dtype=F64), b2D=torch.zeros((2, 3), dtype=F64))
    with pytest.raises(ValueError):
        m.energies(torch.zeros(4, dtype=F64))
    with pytest.raises(ValueError):
        m.energies(torch.zeros(5, dtype=F64), K3D=torch.zeros((2, 3, 3), dtype=F64))
    with pytest.raises(ValueError):
        b.Batch([(m, {"K": torch.zeros(13, dtype=F64), "vol": torch.zeros(1, dtype=F64)}, vla.COEFF_POLY, 1.0, 0.0)])
    with pytest.raises(_LibraryReached):
        m.assemble(K=torch.zeros(13, dtype=F64), M=torch.zeros(13, dtype=F64), vol=torch.zeros(2, dtype=F64))
    with pytest.raises(_LibraryReached):
        m.energies(torch.zeros(5, dtype=F64), K3D=torch.zeros((2, 4, 4), dtype=F64))


def test_gi_inputs_must_agree(b):
    fip = torch.zeros((6, 4, 2), dtype=F64)
    with pytest.raises(ValueError):
        b.gi(fip, [0.25] * 4, torch.zeros(5, dtype=F64))
    with pytest.raises(ValueError):
        b.gi(fip, [0.25] * 4, torch.zeros(6, dtype=F64), normals=torch.zeros((6, 3), dtype=F64))
    with pytest.raises(ValueError):
        b.gi(fip, [0.5] * 2, torch.zeros(6, dtype=F64))
    with pytest.raises(_LibraryReached):
        b.gi(fip, [0.25] * 4, torch.zeros(6, dtype=F64), normals=torch.zeros((6, 2), dtype=F64))


def test_server_requests_must_match_the_element_order(b):
    s = object.__new__(vla.Server)
    s.__dict__.update(_h=None, _keep={}, device=torch.device("cpu"))
    coords = np.zeros((5, 3))
    with pytest.raises(ValueError):
        s.submit(coords, np.zeros((2, 3), dtype=np.int32))
    with pytest.raises(ValueError):
        s.submit(coords, np.zeros((2, 4), dtype=np.int32), faces=np.zeros((4, 2), dtype=np.int32))
    with pytest.raises(_LibraryReached):
        s.submit(coords, np.zeros((2, 4), dtype=np.int32), faces=np.zeros((4, 3), dtype=np.int32))
