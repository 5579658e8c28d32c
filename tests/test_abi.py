"""CPU checks of the C ABI: the library builds, loads, and exports every
function include/sed.h declares, with the documented enum values."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "sed.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sed_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2609_30145_gb300 import build
    build.build()
    from paper_2609_30145_gb300 import _ffi
    return _ffi.load()


def test_every_declared_function_is_exported(lib):
    names = header_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_2609_30145_gb300 import _ffi
    assert sorted(_ffi.SIGNATURES) == header_functions()


def test_enum_values_match_header():
    from paper_2609_30145_gb300 import _ffi
    src = open(os.path.join(ROOT, "include", "sed.h")).read()
    for name, val in [("SED_PREC_FP32", _ffi.PREC_FP32), ("SED_PREC_FP32_SIMT", _ffi.PREC_FP32_SIMT),
                      ("SED_PREC_BF16", _ffi.PREC_BF16), ("SED_EUNSUPPORTED", _ffi.SED_EUNSUPPORTED),
                      ("SED_KEY_GAS_LOGU", _ffi.KEYS.index("gas_logu")),
                      ("SED_KEY_SIGMA_GAL", _ffi.KEYS.index("sigma_gal")),
                      ("SED_KEY_LOG_ERR_SCALE_PHOT", _ffi.KEYS.index("log_err_scale_phot")),
                      ("SED_KEY_LOG_JITTER_SPEC", _ffi.KEYS.index("log_jitter_spec")),
                      ("SED_KEY_FRAC_OBRUN", _ffi.KEYS.index("frac_obrun")),
                      ("SED_KEY_SIGMA_GAS", _ffi.KEYS.index("sigma_gas")),
                      ("SED_KEY_DUST_BINS", _ffi.KEYS.index("dust_bins")),
                      ("SED_KEY_IGM_FACTOR", _ffi.KEYS.index("igm_factor")),
                      ("SED_GAS_SIGMA_SAMPLED", _ffi.GAS_SIGMA_SAMPLED),
                      ("SED_FESC_RUNAWAY_BC", _ffi.FESC_RUNAWAY_BC), ("SED_FESC_PICKET", _ffi.FESC_PICKET),
                      ("SED_FLOOR_ERR_SCALE", _ffi.FLOOR_ERR_SCALE), ("SED_FLOOR_F_CALIB", _ffi.FLOOR_F_CALIB),
                      ("SED_FLOOR_F_DATA", _ffi.FLOOR_F_DATA), ("SED_FLOOR_JITTER", _ffi.FLOOR_JITTER),
                      ("SED_NKEYS", _ffi.NKEYS)]:
        m = re.search(name + r"\b\s*=?\s*(\d+)", src)   # enum "NAME = v" or "#define NAME v"
        assert m and int(m.group(1)) == val, name


def test_status_strings_and_null_args(lib):
    assert lib.sed_status_string(0) == b"ok"
    assert lib.sed_status_string(8) == b"unsupported"
    assert lib.sed_destroy(None) == 1
    assert lib.sed_create(None, 0, 0) == 1
    assert lib.sed_last_error(None) == b"null context"


def test_layout_packing_matches_oracle_layout():
    """The binding's parameter packing and the oracle's agree column by column
    for the documented layout (each side implements it separately)."""
    import numpy as np
    import oracle
    import synth
    from paper_2609_30145_gb300.api import Model
    from paper_2609_30145_gb300 import _ffi
    for zmode in (0, 1):
        for sgal in (0, 1):
            for fp, fs, fe, sgas in ((0, 0, 0, 0), (5, 0, 1, 1), (0, 15, 2, 0), (9, 6, 0, 1)):
                for scheme in (0, 1):
                    ranges = dict(synth.WORKLOADS["tiny_phot_16x4x512"].ranges, sigma_gal=(50.0, 500.0))
                    d = synth.make_theta(5, 7, zmode, ranges, seed=3)
                    if scheme == 1:   # linear SFH scheme: one SFR per bin edge
                        d["sfh"] = synth.edge_sfr(5, 7, seed=3)
                    rng = np.random.default_rng(4)
                    for k in _ffi.KEYS[12:]:
                        d[k] = rng.uniform(-2.0, 0.5, 5)
                    d["frac_obrun"] = rng.uniform(0.0, 1.0, 5)
                    d["sigma_gas"] = rng.uniform(50.0, 400.0, 5)
                    nb = 2 * scheme + fe % 2   # 0..3 age-binned dust laws
                    d["dust_bins"] = rng.uniform(-1.0, 1.5, (5, 2 * nb))
                    igm = (fp + scheme) % 2
                    d["igm_factor"] = rng.uniform(0.5, 1.5, 5)
                    m = Model.__new__(Model)
                    nz = 7 if zmode == 0 else 1
                    # the library's layout: the SFH key has N_T (+1 for the linear
                    # scheme) columns; sigma_gal, each floor term, f_ob and sigma_gas one only
                    # when on; two per age-binned dust law
                    widths = [7 + scheme, nz] + [1] * 9 + [sgal] + [(fp >> k) & 1 for k in range(4)] + \
                             [(fs >> k) & 1 for k in range(4)] + [1 if fe else 0] + [sgas] + [2 * nb] + [igm]
                    offs = list(np.cumsum([0] + widths[:-1]))
                    m.n_param = int(sum(widths))
                    m.offsets = dict(zip(_ffi.KEYS, offs))
                    a = m.pack(d, dtype=np.float64)
                    b = oracle.pack_theta(d, 7, zmode, sample_sigma_gal=sgal, floor_phot=fp, floor_spec=fs,
                                          sfh_scheme=scheme, fesc_geometry=fe, sample_sigma_gas=sgas,
                                          dust_n_bin=nb, use_igm=igm)
                    np.testing.assert_array_equal(a, b)


def test_struct_layouts_match_header(tmp_path):
    """Every descriptor the binding passes by pointer has, field by field, the
    offsets and size a C compiler gives the header's struct."""
    import shutil
    import subprocess
    from paper_2609_30145_gb300 import _ffi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"sed_grid_desc": _ffi.GridDesc, "sed_model_desc": _ffi.ModelDesc,
               "sed_stage_stats": _ffi.StageStats, "sed_server_desc": _ffi.ServerDesc,
               "sed_server_stats": _ffi.ServerStats, "sed_nss_desc": _ffi.NssDesc,
               "sed_nss_result": _ffi.NssResult}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sed.h"', "int main(void) {"]
    want = []
    for cname, cls in structs.items():
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
        want.append(C.sizeof(cls))
        for f, _ in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {f}));')
            want.append(getattr(cls, f).offset)
    for name in ("SED_GRID_COPY_FP32", "SED_GRID_COPY_FP32_SIMT", "SED_GRID_COPY_BF16", "SED_GRID_COPY_FP8",
                 "SED_NOALLOC_SCRATCH_BYTES"):
        lines.append(f'  printf("%zu\\n", (size_t)({name}));')
        want.append(getattr(_ffi, name[4:]))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert got == want
