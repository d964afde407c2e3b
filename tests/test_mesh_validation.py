"""lmood_mesh_create checks its inputs on the host before any device work (CPU only): bad
dimensions, index ranges, inverted or degenerate cells, boundary faces that are not faces of a
cell or carry an unknown tag, batches whose instances share a node."""
import numpy as np
import pytest

import paper_2104_02139_gb300 as L

X2 = np.array([[0.0, 1.0, 1.0, 0.0], [0.0, 0.0, 1.0, 1.0]])
C2 = np.array([[0, 0], [1, 2], [2, 3]], np.int32)  # two counter-clockwise triangles


def _status(f):
    try:
        f()
    except L.LmoodError as e:
        return e.status
    return L.OK


@pytest.fixture(scope="module", autouse=True)
def _built():
    L.build()


def test_bad_cells():
    assert _status(lambda: L.Mesh(4, X2, C2)) == L.ERR_ARG
    assert _status(lambda: L.Mesh(2, X2, C2[[0, 2, 1]])) == L.ERR_MESH  # clockwise: negative area
    assert _status(lambda: L.Mesh(2, X2, np.array([[0], [1], [9]], np.int32))) == L.ERR_MESH
    assert _status(lambda: L.Mesh(2, X2, np.array([[0], [1], [-1]], np.int32))) == L.ERR_MESH
    flat = np.array([[0.0, 1.0, 2.0], [0.0, 0.0, 0.0]])
    assert _status(lambda: L.Mesh(2, flat, np.array([[0], [1], [2]], np.int32))) == L.ERR_MESH
    x3 = np.array([[0.0, 1, 0, 0], [0.0, 0, 1, 0], [0.0, 0, 0, 1]])
    assert _status(lambda: L.Mesh(3, x3, np.array([[0], [2], [1], [3]], np.int32))) == L.ERR_MESH  # inverted tet


def test_bad_boundary_faces():
    bf = np.array([[0, 1], [1, 2]], np.int32)
    assert _status(lambda: L.Mesh(2, X2, C2, bf, np.array([1, 7], np.int32))) == L.ERR_ARG  # unknown tag
    assert _status(lambda: L.Mesh(2, X2, C2, np.array([[0], [7]], np.int32), np.array([1], np.int32))) == L.ERR_MESH
    # (0, 2) is the shared diagonal, a face of two cells: not a boundary face
    assert _status(lambda: L.Mesh(2, X2, C2, np.array([[0], [2]], np.int32), np.array([1], np.int32))) == L.ERR_MESH
    # (1, 3) is no cell's face
    assert _status(lambda: L.Mesh(2, X2, C2, np.array([[1], [3]], np.int32), np.array([1], np.int32))) == L.ERR_MESH
    # the same face twice, in either node order (its nodes would take its traction share twice)
    for dup in (np.array([[0, 0], [1, 1]], np.int32), np.array([[0, 1], [1, 0]], np.int32)):
        assert _status(lambda: L.Mesh(2, X2, C2, dup, np.array([3, 3], np.int32))) == L.ERR_MESH
    x3 = np.array([[0.0, 1, 0, 0], [0.0, 0, 1, 0], [0.0, 0, 0, 1]])
    tet = np.array([[0], [1], [2], [3]], np.int32)
    dup3 = np.array([[0, 2], [1, 0], [2, 1]], np.int32)  # face (0, 1, 2) listed as (0,1,2) and (2,0,1)
    assert _status(lambda: L.Mesh(3, x3, tet, dup3, np.array([1, 4], np.int32))) == L.ERR_MESH


def test_bad_batches():
    # both triangles share nodes 0 and 2, so they cannot be two instances
    assert _status(lambda: L.Mesh(2, X2, C2, cell_inst=np.array([0, 1], np.int32), n_inst=2)) == L.ERR_MESH
    assert _status(lambda: L.Mesh(2, X2, C2, cell_inst=np.array([0, 5], np.int32), n_inst=2)) == L.ERR_ARG


def test_no_device_is_a_cuda_error():
    """A valid mesh on a machine without a usable GPU fails cleanly with LMOOD_ERR_CUDA."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    assert _status(lambda: L.Mesh(2, X2, C2)) == L.ERR_CUDA
