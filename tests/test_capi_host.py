"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/sha3gb.h declares, carries the round constants and rho
offsets the standard fixes, and rejects bad arguments before touching CUDA."""
import ctypes

import pytest

from paper_1902_05320_gb300 import binding, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def test_exports_every_declared_function(lib):
    names = binding.declared_functions()
    assert {"keccak_batch", "keccak_batch_uniform", "merkle_sha3_256", "keccak_last_error"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name


def test_round_constants_match_oracle_lfsr(lib, oracle_mod):
    # Definition 5 / Eq. 8: the kernels' immediates equal rc() regenerated by
    # the oracle's FIPS 202 Algorithm 5 register.
    assert binding.round_constants() == [oracle_mod.round_constant(6, ir) for ir in range(24)]


def test_rho_offsets_match_oracle_walk(lib, oracle_mod):
    want = [oracle_mod.rho_offset(64, i % 5, i // 5) for i in range(25)]
    assert binding.rho_offsets() == want


def test_version(lib):
    assert "sm_103a" in binding.version()


def test_argument_errors_are_returned_before_any_cuda_call(lib):
    # Null pointers with n > 0, unknown variants and SHA3 output sizes other
    # than the digest size are KB_ERR_INVALID; n = 0 is a no-op.
    assert lib.keccak_batch_uniform(None, 64, 64, 1, 32, None, 0, None) == binding.KB_OK
    assert lib.keccak_batch_uniform(None, 64, 64, 1, 32, None, 5, None) == binding.KB_ERR_INVALID
    assert lib.keccak_batch_uniform(None, 64, 64, 6, 32, None, 0, None) == binding.KB_ERR_INVALID
    assert lib.keccak_batch_uniform(None, 64, 64, 1, 31, None, 0, None) == binding.KB_ERR_INVALID
    assert lib.keccak_batch_uniform(None, 64, 0, 4, 0, None, 0, None) == binding.KB_OK
    assert lib.keccak_batch(None, None, None, None, None, None, 0, None) == binding.KB_OK
    assert lib.keccak_batch(None, None, None, None, None, None, 3, None) == binding.KB_ERR_INVALID
    assert lib.keccak_batch_uniform_host(None, 8, 8, 1, 32, None, 2, None) == binding.KB_ERR_INVALID
    root = (ctypes.c_uint8 * 32)()
    assert lib.merkle_sha3_256(None, 0, 8, ctypes.addressof(root), None) == binding.KB_ERR_INVALID
    assert lib.merkle_sha3_256(1 << 20, 4, 0, ctypes.addressof(root), None) == binding.KB_ERR_INVALID
    assert lib.merkle_sha3_256_levels(1 << 20, 0, 8, 1 << 20, None) == binding.KB_ERR_INVALID
    # Overflowing sizes.
    assert lib.keccak_batch_uniform(1 << 20, 1 << 40, 64, 1, 32, 1 << 20, 1 << 30, None) == binding.KB_ERR_INVALID
    # The bounded-wait check: a limit of 0 or above 2 s, or arrive not 0/1.
    assert lib.sha3gb_wait_timeout_probe(0, 0, None) == binding.KB_ERR_INVALID
    assert lib.sha3gb_wait_timeout_probe(2_000_000_001, 0, None) == binding.KB_ERR_INVALID
    assert lib.sha3gb_wait_timeout_probe(1000, 2, None) == binding.KB_ERR_INVALID


def test_merkle_node_count(lib, oracle_mod):
    for n in (0, 1, 2, 3, 5, 7, 8, 9, 1000, 524288):
        assert binding.merkle_node_count(n) == oracle_mod.merkle_node_count(n)


def test_tuning_knobs_validate_values(lib):
    keys = range(binding.KB_TUNE_KEYS)
    saved = [binding.keccak_tune_get(k) for k in keys]
    try:
        assert saved[0] == binding.KB_REP_PLAIN and saved[1] == binding.KB_SCHEDULE_QUEUE
        assert saved[binding.KB_TUNE_QUEUE_STAGING] == 0 and saved[binding.KB_TUNE_QUEUE_WARP_MESSAGES] == -1
        for key, bad in ((0, 2), (1, 4), (2, 3), (3, -1), (4, 1), (4, 7), (5, 33), (6, 3), (7, 2), (8, 5), (8, -1),
                         (9, -2), (9, 1 << 32), (10, 0), (99, 0)):
            assert lib.keccak_tune_set(key, bad) == binding.KB_ERR_INVALID
        assert binding.keccak_tune_get(99) == -1
        for key, good in ((0, 1), (1, 0), (2, 0), (3, 0), (4, 6), (5, 3), (6, 1), (7, 1), (8, 4), (9, 0), (9, 608)):
            binding.keccak_tune_set(key, good)
            assert binding.keccak_tune_get(key) == good
    finally:
        for k, v in zip(keys, saved):
            binding.keccak_tune_set(k, v)


def test_binding_constants_match_the_header():
    # Every numeric #define and enum value of the header, as the binding has it.
    import os
    import re

    text = open(os.path.join(os.path.dirname(__file__), "..", "include", "sha3gb.h")).read()
    found = {}
    for name, value in re.findall(r"#define\s+(KB_\w+)\s+(-?(?:0x[0-9a-fA-F]+|\d+))u?\b", text):
        found[name] = int(value, 0)
    for name, value in re.findall(r"\b(KB_\w+)\s*=\s*(-?\d+)", text):
        found[name] = int(value)
    assert len(found) > 30
    missing = [k for k in found if not hasattr(binding, k)]
    assert not missing, missing
    wrong = {k: (v, getattr(binding, k)) for k, v in found.items() if getattr(binding, k) != v}
    assert not wrong, wrong


def test_header_is_plain_c(tmp_path):
    # The boundary is a C ABI: the header compiles as C99 and as C++ on its
    # own (no CUDA, torch or C++ types), warnings as errors.
    import os
    import subprocess

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "use.c"
    src.write_text('#include "sha3gb.h"\n'
                   'int use(const uint8_t *m, uint8_t *d, void *s) {\n'
                   '    int rc = keccak_batch_uniform(m, 64, 64, KB_SHA3_256, 32, d, 1, s);\n'
                   '    return rc == KB_OK ? keccak_last_error(s) : rc;\n'
                   '}\n')
    inc = os.path.join(root, "include")
    for cmd in (["gcc", "-std=c99", "-pedantic"], ["g++", "-std=c++17", "-x", "c++"]):
        r = subprocess.run(cmd + ["-Wall", "-Wextra", "-Werror", "-I", inc, "-c", str(src), "-o",
                                  str(tmp_path / "use.o")], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_binding_signatures_cover_the_header():
    # Every function the header declares has a ctypes signature in the
    # binding, with as many arguments as the prototype.
    import re

    text = open(binding.HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    protos = {}
    for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_ \*]*?)\b([a-z_][a-z0-9_]*)\s*\(([^;{]*?)\)\s*;", text):
        name, params = m.group(2), " ".join(m.group(3).split())
        if name in binding.declared_functions():
            protos[name] = 0 if params in ("", "void") else params.count(",") + 1
    assert set(protos) == set(binding.declared_functions())
    from paper_1902_05320_gb300 import serve

    lib = serve._lib()  # the binding's signatures plus the server's
    for name, nargs in protos.items():
        fn = getattr(lib, name)
        assert fn.argtypes is not None and len(fn.argtypes) == nargs, name


def test_struct_layouts_match_the_header(tmp_path):
    # The ctypes mirrors of the header's structs (kb_queue_config,
    # kb_server_config, kb_server_stats) must have the C compiler's size and
    # field offsets, or the library would read and write the wrong bytes.
    import shutil
    import subprocess

    from paper_1902_05320_gb300 import serve

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {"kb_queue_config": binding.QueueConfig, "kb_server_config": serve.ServerConfig,
               "kb_server_stats": serve.ServerStats}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "sha3gb.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'    printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = str(binding.HEADER).rsplit("/", 1)[0]
    subprocess.run([cc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(ln.split()[:2]): int(ln.split()[2]) for ln in out if ln.strip()}
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)


def test_readme_c_example_compiles(tmp_path):
    # The C usage example in README.md compiles against the header and the
    # CUDA runtime's header (warnings as errors), so the documented calls
    # keep matching the ABI.
    import os
    import re
    import shutil
    import subprocess

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    blocks = re.findall(r"```c\n(.*?)```", open(os.path.join(root, "README.md")).read(), flags=re.S)
    assert blocks, "README.md has no C example"
    cuda_inc = next((d for d in ("/usr/local/cuda/include",) if os.path.exists(os.path.join(d, "cuda_runtime.h"))),
                    None)
    if cuda_inc is None or shutil.which("gcc") is None:
        pytest.skip("no CUDA headers or C compiler")
    for k, code in enumerate(blocks):
        src = tmp_path / f"example{k}.c"
        src.write_text(code)
        r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(root, "include"),
                            "-I", cuda_inc, "-c", str(src), "-o", str(tmp_path / f"example{k}.o")],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
