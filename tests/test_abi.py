"""The C-ABI library builds, loads without a GPU and exports what include/mbe.h declares."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mbe.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mbe_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("mbe_graph_create", "mbe_graph_destroy", "mbe_enumerate", "mbe_enumerate_batch",
                     "mbe_status_string", "mbe_default_options"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_2401_05039_gb300 as m
    lib = m.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    nm = subprocess.run(["nm", "-D", "--defined-only", m.library_path()], capture_output=True, text=True).stdout
    for n in declared_functions():
        assert re.search(rf"\bT {n}$", nm, flags=re.M), n


def test_host_only_calls_without_gpu():
    import paper_2401_05039_gb300 as m
    lib = m.load()
    assert lib.mbe_status_string(0) == b"MBE_OK"
    assert lib.mbe_status_string(4) == b"MBE_ERR_ARENA_FULL"
    assert lib.mbe_status_string(99) == b"MBE_ERR_UNKNOWN"
    o = m.options()
    assert o.steal == 1 and o.root_end == -1 and o.emit == 0
    assert lib.mbe_default_options(None) == 1
    assert lib.mbe_enumerate(None, None, None, None, None) == 1


def test_struct_layouts_match_c(tmp_path):
    import paper_2401_05039_gb300 as m
    src = tmp_path / "layout.c"
    src.write_text(f'''
#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
int main(void) {{
  printf("%zu %zu %zu\\n", sizeof(mbe_options), sizeof(mbe_result), sizeof(mbe_biclique_buffer));
  printf("%zu %zu %zu %zu %zu\\n", offsetof(mbe_options, arena_bytes), offsetof(mbe_options, model),
         offsetof(mbe_options, per_root), offsetof(mbe_options, n_exec), offsetof(mbe_options, min_l));
  printf("%zu %zu %zu\\n", offsetof(mbe_result, device_ms), offsetof(mbe_result, status),
         offsetof(mbe_result, n_donations));
  printf("%zu %zu %zu %zu %zu\\n", offsetof(mbe_options, layout), sizeof(mbe_class_params),
         offsetof(mbe_class_params, layout), offsetof(mbe_class_params, tuned_ms),
         offsetof(mbe_class_params, default_ms));
  printf("%zu\\n", offsetof(mbe_options, prune));
  return 0;
}}''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split()
    vals = [int(x) for x in out]
    O, R, B = m.Options, m.Result, m.BicliqueBuffer
    assert vals[:3] == [ctypes.sizeof(O), ctypes.sizeof(R), ctypes.sizeof(B)]
    assert vals[3:8] == [O.arena_bytes.offset, O.model.offset, O.per_root.offset, O.n_exec.offset, O.min_l.offset]
    assert vals[8:11] == [R.device_ms.offset, R.status.offset, R.n_donations.offset]
    C = m.ClassParams
    assert vals[11:16] == [O.layout.offset, ctypes.sizeof(C), C.layout.offset, C.tuned_ms.offset, C.default_ms.offset]
    assert vals[16] == O.prune.offset


def test_compress_helper_matches_bit_gather(tmp_path):
    # the device bit-compression helper, compiled for the host
    src = tmp_path / "comp.cpp"
    src.write_text('''
#include "%s"
#include <cstdio>
#include <random>
static uint64_t gather(uint64_t x, uint64_t m){uint64_t r=0;int k=0;for(int i=0;i<64;i++) if(m>>i&1){r|=((x>>i)&1ULL)<<k;k++;}return r;}
int main(){std::mt19937_64 g(5);long bad=0;for(int t=0;t<300000;t++){uint64_t m=g(),x=g();if(t%%3==1)m&=g();if(t%%3==2)m|=g();
 if(t%%97==0)m=0;if(t%%89==0)m=~0ULL;mbe::CompressMasks c=mbe::compress_prepare(m);if(mbe::compress_apply(x,c)!=gather(x,m))bad++;mbe::CompressMasks c2=mbe::compress_prepare_rolled(m);if(mbe::compress_apply(x,c2)!=gather(x,m))bad++;}
 printf("%%ld\\n",bad);return 0;}''' % os.path.join(ROOT, "paper_2401_05039_gb300", "csrc", "mbe_bits.h"))
    exe = tmp_path / "comp"
    subprocess.check_call(["g++", "-O2", "-std=c++17", str(src), "-o", str(exe)])
    assert subprocess.check_output([str(exe)], text=True).strip() == "0"


def test_device_hash_matches_oracle_hash(tmp_path):
    # the library's SplitMix64 (host-compiled) against the oracle's, on 10^5 inputs
    import oracle
    src = tmp_path / "sm.cpp"
    src.write_text('''
#include "%s"
#include <cstdio>
int main(){unsigned long long z=0x1234567ULL;for(int i=0;i<100000;i++){z=z*6364136223846793005ULL+1442695040888963407ULL;
 printf("%%llu\\n",(unsigned long long)mbe::splitmix(z));}return 0;}''' % os.path.join(
        ROOT, "paper_2401_05039_gb300", "csrc", "mbe_bits.h"))
    exe = tmp_path / "sm"
    subprocess.check_call(["g++", "-O2", "-std=c++17", str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)], text=True).split()]
    z = 0x1234567
    M = (1 << 64) - 1
    exp = []
    for _ in range(100000):
        z = (z * 6364136223846793005 + 1442695040888963407) & M
        exp.append(oracle.sm(z))
    assert got == exp


def test_batch_size_classes():
    import paper_2401_05039_gb300 as m
    assert m.batch_class(16, 16, 10) == 0
    assert m.batch_class(16, 16, 100) == 1          # density >= 0.1
    assert m.batch_class(200, 16, 10) == 4
    assert m.batch_class(16, 600, 10) == 2
    assert m.batch_class(512, 2048, 200000) == 7


def _bad_host_graphs():
    """Host graphs whose offsets or ids fall outside the arrays (never sent to a device)."""
    import numpy as np
    from tests import helpers as H
    g = H.random_graph(np.random.default_rng(1), 10, 12, 0.4)
    arrs = [np.ascontiguousarray(a, dtype=np.int32).copy() for a in (g.u_off, g.u_adj, g.v_off, g.v_adj)]
    cases = []

    def case(name, k, idx, val):
        a = [x.copy() for x in arrs]
        a[k][idx] = val
        cases.append((name, a))

    case("u id = nV", 1, 0, g.nV)
    case("u id negative", 1, 3, -5)
    case("v id = nU", 3, 2, g.nU)
    case("u offset past nE", 0, 4, g.nE + 7)
    case("u offsets decrease", 0, 5, int(arrs[0][4]) - 1 if arrs[0][4] > 0 else -1)
    case("v offset negative", 2, 3, -1)
    case("u_off[0] != 0", 0, 0, 1)
    case("v_off[nV] != nE", 2, g.nV, g.nE - 1)
    return g, cases


def test_host_graph_out_of_range_rejected_before_any_device_work():
    # host input is range-checked on the host: MBE_ERR_INVALID_GRAPH comes
    # back before any CUDA call, so this runs without a GPU
    import paper_2401_05039_gb300 as m
    lib = m.load()
    g, cases = _bad_host_graphs()
    for name, (uo, ua, vo, va) in cases:
        h = ctypes.c_void_p()
        st = lib.mbe_graph_create(g.nU, g.nV, g.nE, uo.ctypes.data, ua.ctypes.data, vo.ctypes.data, va.ctypes.data,
                                  0, None, ctypes.byref(h))
        assert st == 2 and not h.value, name


def test_host_batch_out_of_range_rejected_before_any_device_work():
    # the same corruptions in the second graph of a packed batch (host arrays)
    import synth
    import paper_2401_05039_gb300 as m
    g, cases = _bad_host_graphs()
    for name, (uo, ua, vo, va) in cases:
        b = synth.pack([g, g])
        e0, us, vs = int(b.edge_off[1]), int(b.u_off_start[1]), int(b.v_off_start[1])
        b.u_off[us:us + g.nU + 1] = uo
        b.v_off[vs:vs + g.nV + 1] = vo
        b.u_adj[e0:e0 + g.nE] = ua
        b.v_adj[e0:e0 + g.nE] = va
        per, tot = m.enumerate_batch(b, check=False)
        assert tot.status == 2, name
