"""The persistent tuning cache (cpb_tuning_save / cpb_tuning_load): host-only,
no GPU needed when the device name is given."""
import pytest

cpb = pytest.importorskip("paper_2206_07896_gb300")


@pytest.fixture()
def L():
    return cpb.Library(cpb.build.lib_path("libcpb.so"))


def test_save_load_roundtrip(L, tmp_path):
    t1 = {"k": 8, "chunk_rows": 512, "warps_per_block": 4, "variant": 1, "stages": 4}
    t2 = {"k": 3, "chunk_rows": 96, "warps_per_block": 2, "variant": 0, "stages": 2}
    L.cpb_set_tuning(8191, 8189, cpb.CPB_F32, cpb.CPB_PERIODIC, t1)
    L.cpb_set_tuning(1001, 37, cpb.CPB_BF16_KAHAN, cpb.CPB_DIRICHLET0, t2)
    path = tmp_path / "tune.txt"
    L.cpb_tuning_save(str(path), "Test GPU A")
    lines = path.read_text().splitlines()
    assert any(ln.startswith("cpb-tuning 1 Test_GPU_A 8191 8189 0 1 8 512 4 1 4") for ln in lines)
    fresh = cpb.Library(cpb.build.lib_path("libcpb_nofma.so"))   # another process-wide cache
    assert fresh.cpb_lookup_tuning(1001, 37, cpb.CPB_BF16_KAHAN, cpb.CPB_DIRICHLET0) is None
    assert fresh.cpb_tuning_load(str(path), "Test GPU B") == 0      # other device: skipped
    assert fresh.cpb_lookup_tuning(8191, 8189, cpb.CPB_F32, cpb.CPB_PERIODIC) is None
    assert fresh.cpb_tuning_load(str(path), "Test GPU A") == len(lines)
    assert fresh.cpb_lookup_tuning(8191, 8189, cpb.CPB_F32, cpb.CPB_PERIODIC) == t1
    assert fresh.cpb_lookup_tuning(1001, 37, cpb.CPB_BF16_KAHAN, cpb.CPB_DIRICHLET0) == t2
    assert fresh.cpb_get_tuning(1001, 37, cpb.CPB_BF16_KAHAN, cpb.CPB_DIRICHLET0) == t2


def test_bad_lines_and_missing_file_are_rejected(L, tmp_path):
    with pytest.raises(cpb.CpbError) as e:
        L.cpb_tuning_load(str(tmp_path / "missing.txt"), "X")
    assert e.value.status == cpb.CPB_ERR_INVALID_VALUE
    bad = tmp_path / "bad.txt"
    bad.write_text("cpb-tuning 1 X 64 64 0 0 4 256 1 1 2\n"
                   "cpb-tuning 1 X 64 64 0 0 9 256 1 1 2\n")     # depth 9 is not a valid tuning
    with pytest.raises(cpb.CpbError) as e:
        L.cpb_tuning_load(str(bad), "X")
    assert e.value.status == cpb.CPB_ERR_INVALID_VALUE
    assert L.cpb_lookup_tuning(64, 64, cpb.CPB_F32, cpb.CPB_DIRICHLET0)["k"] == 4   # the line before stays
    junk = tmp_path / "junk.txt"
    junk.write_text("not a tuning line\n")
    with pytest.raises(cpb.CpbError):
        L.cpb_tuning_load(str(junk), "X")
