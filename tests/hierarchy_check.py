"""Shared GPU-vs-oracle hierarchy comparison for the parity tests."""
import numpy as np


def check_hierarchy(amg, h, H):
    """Every level of the GPU hierarchy h equals the oracle's H bit for bit:
    matrices, aggregates of both passes, intermediate products, colourings,
    ILU(0) factors."""
    nlev = amg.amg_num_levels(h)
    assert nlev == H.nlev
    for l in range(nlev):
        gi = amg.amg_get_level_info(h, l)
        lo = H.levels[l]
        assert gi["n"] == lo["n"] and gi["nnz"] == lo["nnz"] and bool(gi["dense"]) == lo["dense"]
        rp, ci, v = amg.amg_get_matrix(h, l)
        M = H.matrix(l)
        assert np.array_equal(rp, M.row_ptr) and np.array_equal(ci, M.col)
        assert np.array_equal(v, M.val), f"level {l} values differ"
        if l + 1 < nlev:
            npass = lo["npass"]
            assert np.array_equal(amg.amg_get_aggregates(h, l, 0), H.agg(l, 0)), f"level {l} aggregates"
            for p in range(1, npass + 1):
                assert np.array_equal(amg.amg_get_aggregates(h, l, p), H.agg(l, p)), f"level {l} pass {p}"
            for p in range(1, npass):
                rp1, ci1, v1 = amg.amg_get_pass_matrix(h, l, p)
                M1 = H.mid(l, p)
                assert np.array_equal(rp1, M1.row_ptr) and np.array_equal(ci1, M1.col) and \
                    np.array_equal(v1, M1.val), f"level {l} pass {p} product"
        if not lo["dense"]:
            assert np.array_equal(amg.amg_get_colors(h, l), H.colors(l)), f"level {l} colours"
            assert np.array_equal(amg.amg_get_ilu(h, l), H.lu(l)), f"level {l} ILU(0)"
