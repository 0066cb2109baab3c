"""Row-block partition on the GPU (assembly split by rows for several GPUs):
vla_partition_rows selects the elements with a node in a block of rows
(bit-exact against the definition), and the sub-mesh handles of all blocks
(vla_mesh_create_rows), each assembled on its own, give the whole mesh's CSR
pattern and K, M values when their owned rows are concatenated -- bit for bit
against the whole-mesh GPU assembly (same summation order) and within the
FP64 tolerance against the oracle.  The blocks run one after another on one
GPU here; on several GPUs each would run on its own with no exchange."""
import numpy as np
import pytest
import torch

import meshgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vla():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2404_16039_gb300 as v
    v.lib()
    return v


def _blocks(nn, n):
    return [(nn * r // n, nn * (r + 1) // n) for r in range(n)]


@pytest.mark.parametrize("dim,order,n,parts", [(3, 1, 7, 3), (2, 2, 9, 2), (3, 2, 3, 4), (2, 1, 20, 5)])
def test_row_blocks_concatenate_to_the_whole_mesh(vla, dim, order, n, parts):
    m = meshgen.make_mesh(dim, n, order=order, jitter=0.1, seed=12)
    c, e, f = (torch.from_numpy(m.coords).cuda(), torch.from_numpy(m.elems).cuda(),
               torch.from_numpy(m.faces).cuda())
    whole = vla.Mesh(c, e, f, order=order)
    ref = oracle.assemble(dim, order, m.nn, m.elems, m.coords, 0.7, 1.3)
    for prec in (vla.PREC_FP64, vla.PREC_MIXED):
        w = whole.assemble(0.7, 1.3, precision=prec)
        rps, cis, Ks, Ms, nfb = [], [], [], [], 0
        for r0, r1 in _blocks(m.nn, parts):
            ids = vla.partition_rows(e, r0, r1).cpu().numpy()
            touch = np.nonzero(((m.elems >= r0) & (m.elems < r1)).any(axis=1))[0]
            assert np.array_equal(ids, touch)                       # integer work: bit-exact
            sub = vla.Mesh(c, e, f, order=order, rows=(r0, r1))
            assert sub.ne == len(touch)
            o = sub.assemble(0.7, 1.3, precision=prec)
            rp, ci, K, M = sub.block((o["K"], o["M"]))
            base = rps[-1][-1] if rps else 0
            rps.append((rp.cpu().numpy() + base) if not rps else (rp.cpu().numpy()[1:] + base))
            cis.append(ci.cpu().numpy())
            Ks.append(K)
            Ms.append(M)
            # volumes of the sub-mesh's elements are those elements' volumes in the whole mesh
            assert torch.equal(o["vol"], w["vol"][torch.from_numpy(touch).cuda()])
            nfb += sub.nfb
            sub.close()
        rp = np.concatenate(rps)
        ci = np.concatenate(cis)
        assert np.array_equal(rp, ref["row_ptr"]) and np.array_equal(ci, ref["col_idx"])
        K, M = torch.cat(Ks), torch.cat(Ms)
        assert torch.equal(K, w["K"]) and torch.equal(M, w["M"])    # same terms, same order, same bits
        assert nfb == m.nfb                                          # the facets are split among the blocks
        if prec == vla.PREC_FP64:
            rows = np.repeat(np.arange(m.nn), np.diff(ref["row_ptr"]))
            for got, r in ((K.cpu().numpy(), ref["K"]), (M.cpu().numpy(), ref["M"])):
                rowmax = np.zeros(m.nn)
                np.maximum.at(rowmax, rows, np.abs(r))
                assert np.all(np.abs(got - r) <= 1e-12 * np.maximum(np.abs(r), rowmax[rows]))
    whole.close()


def test_partition_arguments(vla):
    m = meshgen.kuhn_cube(3, jitter=0.1, seed=1)
    c, e = torch.from_numpy(m.coords).cuda(), torch.from_numpy(m.elems).cuda()
    assert vla.partition_rows(e, 5, 5).numel() == 0              # an empty block selects nothing
    for bad in ((-1, 4), (4, 2), (0, m.nn + 1)):
        with pytest.raises(vla.VlaError):
            vla.Mesh(c, e, rows=bad)
