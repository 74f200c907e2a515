"""CPU-side checks of the C ABI library: it loads and exports every entry
point include/palmad.h declares; host-side argument and option rules that
need no GPU."""
import ctypes
import os
import re

import numpy as np

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "palmad.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(palmad_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2304_01660_gb300 import _build, palmad
    _build.build()
    return palmad.load()


def test_header_declares_the_boundary():
    names = _declared()
    for want in ["palmad_create", "palmad_destroy", "palmad_find_discords", "palmad_find_discords_device",
                 "palmad_find_discords_batch", "palmad_drag", "palmad_last_error", "palmad_default_options",
                 "palmad_get_stats", "palmad_version", "palmad_autotune"]:
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_default_options_and_version(lib):
    from paper_2304_01660_gb300 import palmad
    o = palmad.palmad_default_options()
    assert o.struct_size == ctypes.sizeof(palmad.Options)
    assert o.exclusive_topk == 1 and o.band_rel == pytest.approx(1e-3)
    # the documented defaults: FP32, plain form, automatic caps and segments,
    # nearest-neighbour distance
    assert (o.precision, o.batch_lengths, o.select_cap, o.pool_slots, o.refine_seg, o.knn_k) == (0, 0, 0, 0, 0, 0)
    assert (o.direct_below, o.tc_seed_min, o.seed_rows_max, o.profile) == (0, 0, 0, 0)
    # witness hints on, the batched margins as documented, no autotuning
    assert (o.no_hints, o.spec_scale, o.autotune) == (0, 0, 0)
    assert palmad.palmad_default_options(knn_k=3, batch_lengths=16).knn_k == 3
    with pytest.raises(KeyError):
        palmad.palmad_default_options(no_such_option=1)
    assert lib.palmad_default_options(None) == -1
    assert "sm_103a" in palmad.palmad_version()


def test_struct_layouts_match_header(tmp_path):
    """ctypes mirrors of palmad_options / palmad_stats match the C layout
    (a C probe compiled against the header prints sizes and offsets)."""
    import subprocess
    from paper_2304_01660_gb300 import palmad
    probe = tmp_path / "probe.c"
    probe.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "palmad.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(palmad_options),
         offsetof(palmad_options, band_rel),
         offsetof(palmad_options, profile), sizeof(palmad_stats), offsetof(palmad_stats, max_fp32_rho_err),
         offsetof(palmad_stats, kernel_ms), offsetof(palmad_stats, refine_flops),
         offsetof(palmad_options, direct_below), offsetof(palmad_options, refine_seg),
         offsetof(palmad_stats, seed_flops), offsetof(palmad_options, knn_k),
         offsetof(palmad_options, autotune), offsetof(palmad_stats, tune_ms), offsetof(palmad_stats, hint_kills),
         sizeof(palmad_tune_report), offsetof(palmad_tune_report, default_ms));
  return 0;
}
""")
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(probe), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    O, S, R = palmad.Options, palmad.Stats, palmad.TuneReport
    assert got == [ctypes.sizeof(O), O.band_rel.offset, O.profile.offset, ctypes.sizeof(S),
                   S.max_fp32_rho_err.offset, S.kernel_ms.offset, S.refine_flops.offset,
                   O.direct_below.offset, O.refine_seg.offset, S.seed_flops.offset, O.knn_k.offset,
                   O.autotune.offset, S.tune_ms.offset, S.hint_kills.offset, ctypes.sizeof(R), R.default_ms.offset]


def test_every_field_offset_matches_header(tmp_path):
    """Every field of the ctypes mirrors (palmad_options, palmad_stats,
    palmad_tune_report) sits at the offset the C compiler gives it."""
    import subprocess
    from paper_2304_01660_gb300 import palmad
    mirrors = {"palmad_options": palmad.Options, "palmad_stats": palmad.Stats,
               "palmad_tune_report": palmad.TuneReport}
    lines = []
    for cname, cls in mirrors.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    probe = tmp_path / "fields.c"
    probe.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "palmad.h"\nint main(void) {\n'
                     + "\n".join(lines) + "\n  return 0;\n}\n")
    exe = tmp_path / "fields"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(probe), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(line.split() for line in out if line)
    for cname, cls in mirrors.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(cls, fname).offset, f"{cname}.{fname}"


def test_tensor_core_options_default_to_automatic(lib):
    from paper_2304_01660_gb300 import palmad
    o = palmad.palmad_default_options()
    # refine form split for long windows, strip height, MMA survivor group,
    # column chunks and the tensor-core kernel form all start automatic
    assert (o.direct_below_long, o.refine_rows, o.tc_group, o.tc_chunks, o.tc_form) == (0, 0, 0, 0, 0)


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.palmad_create(ctypes.byref(h), 0, None) != 0
    assert not h.value


def test_schedule_inputs_reads_the_kth_or_last_pick():
    idx = np.array([[4, 9, 2], [4, 9, -1], [-1, -1, -1]])
    nn = np.array([[3.0, 2.5, 2.0], [3.0, 2.5, 0.0], [0.0, 0.0, 0.0]])
    from paper_2304_01660_gb300 import palmad
    assert palmad.schedule_inputs(idx, nn).tolist() == [2.0, 2.5, 0.0]
