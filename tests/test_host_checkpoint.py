"""BVH checkpoints (sc_bvh_save / sc_bvh_load): a loaded BVH equals the
built one array for array and gives the same device image; damaged files
are refused with SC_ERR_IO."""
import numpy as np
import pytest

from paper_2305_08343_gb300 import subcull as sc


@pytest.mark.parametrize("R,comp", [(0, 0), (6, 0), (6, 1), (4, 1)])
def test_round_trip(hair_small, tmp_path, R, comp):
    tris, _ = hair_small
    b = sc.sc_bvh_build(tris, R, comp, skip_bits=150 if R == 6 else 0)
    p = str(tmp_path / "bvh.ck")
    sc.sc_bvh_save(b, p)
    c = sc.sc_bvh_load(p)
    ia, ib = b.info(), c.info()
    for f in ("num_tris", "num_nodes", "max_depth", "grid_res", "compress", "L", "clut_entries",
              "eps"):
        assert getattr(ia, f) == getattr(ib, f), f
    assert list(ia.root_box) == list(ib.root_box)
    ea, eb = b.export(), c.export()
    assert ea.keys() == eb.keys()
    for k in ea:
        assert np.array_equal(ea[k], eb[k]), k
    if R:
        for lay in (sc.SC_LAYOUT_MASKED, sc.SC_LAYOUT_MASKED_COMPACT):
            assert sc.sc_bvh_device_bytes(b, lay) == sc.sc_bvh_device_bytes(c, lay)
    # saving the loaded BVH reproduces the file byte for byte
    p2 = str(tmp_path / "bvh2.ck")
    sc.sc_bvh_save(c, p2)
    assert open(p, "rb").read() == open(p2, "rb").read()


def test_damaged_files_are_refused(hair_small, tmp_path):
    tris, _ = hair_small
    b = sc.sc_bvh_build(tris, 6, 1)
    p = tmp_path / "bvh.ck"
    sc.sc_bvh_save(b, str(p))
    data = bytearray(p.read_bytes())
    for name, blob in (("flip", data[:100] + bytes([data[100] ^ 1]) + data[101:]),
                       ("truncated", data[: len(data) // 2]), ("empty", b""),
                       ("magic", b"XXXXXXXX" + data[8:])):
        q = tmp_path / f"{name}.ck"
        q.write_bytes(bytes(blob))
        with pytest.raises(sc.SubcullError) as e:
            sc.sc_bvh_load(str(q))
        assert e.value.code == sc.SC_ERR_IO, name
    with pytest.raises(sc.SubcullError) as e:
        sc.sc_bvh_load(str(tmp_path / "missing.ck"))
    assert e.value.code == sc.SC_ERR_IO
