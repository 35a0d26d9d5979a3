"""Checkpoint files are checked on the host before anything is restored: a
file written in the library's format (version 3) by this test passes
gmcs_checkpoint_info with its counts, and every inconsistency a truncated or
corrupted file can carry -- a table or occupancy size that disagrees with its
lattice, a storage type that does not match the config, a config the library
would not accept, a missing or extra byte, an absurd size -- is refused with
GMCS_E_IO without any allocation. No GPU is needed."""
import ctypes as C
import struct

import numpy as np
import pytest

import paper_2504_18056_b300 as g

MAGIC = b"GMCSCKPT"


class Header(C.Structure):
    _fields_ = [("magic", C.c_char * 8), ("version", C.c_uint32), ("frame", C.c_uint32), ("cfg", g.Config),
                ("P", C.c_int32), ("K", C.c_int32), ("path_now", C.c_double), ("odo", C.c_double * 12)]


class TableHead(C.Structure):
    _fields_ = [("dtype", C.c_int32), ("layout", C.c_int32), ("grid", g.Grid), ("bytes", C.c_uint64)]


def grid(origin, h, n):
    gr = g.Grid()
    for a in range(3):
        gr.origin[a] = origin[a]
        gr.n[a] = n[a]
    gr.h = h
    return gr


def write(path, P=5, tables=((0, (4, 3, 2)),), cfg=None, frame=7, tweak=None):
    """A checkpoint with P particles and one field table (dtype, vertex counts)
    per entry; tweak(name, obj) may alter a header before it is written."""
    cfg = cfg or g.default_config()
    h = Header()
    h.magic = MAGIC
    h.version = 3
    h.frame = frame
    h.cfg = cfg
    h.P = P
    h.K = len(tables)
    h.path_now = 1.5
    for e in range(12):
        h.odo[e] = 1.0 if e % 5 == 0 else 0.0
    if tweak:
        tweak("header", h)
    out = bytearray(bytes(h))
    out += np.zeros((P, 12), np.float32).tobytes() + np.full(P, -np.log(P)).tobytes()
    for dt, n in tables:
        th = TableHead()
        th.dtype = dt
        th.layout = cfg.table_layout if dt != 3 else 0
        th.grid = grid((0.0, 0.0, 0.0), 0.2, n)
        rec = 48 if dt == 3 else (32 if dt == 0 else 16)
        if th.layout == g.LAYOUT_COLUMNS:
            # column directory (one run of two cells in every column), then the records
            ncol = (n[0] - 1) * (n[1] - 1)
            dirb = (ncol * 8 + 255) // 256 * 256
            d = np.zeros(dirb // 4, np.uint32)
            d[0:2 * ncol:2] = np.arange(ncol) * 2          # first record of the column
            d[1:2 * ncol:2] = 0 | (2 << 16)                # zlo 0, two cells
            if tweak:
                tweak("dir", d)
            body = d.tobytes() + bytes(2 * ncol * rec)
        else:
            cells = int(np.prod(n)) if dt == 3 else int(np.prod([v - 1 for v in n]))
            body = bytes(cells * rec)
        th.bytes = len(body)
        if tweak:
            tweak("table", th)
        out += bytes(th) + body
        og = grid((-1.0, -1.0, -1.0), 1.0, (3, 3, 2))
        occ = 3 * 3 * 2
        if tweak:
            tweak("occ", og)
        out += bytes(og) + struct.pack("<Q", occ) + bytes(occ)
        out += struct.pack("<d", 0.5) + np.zeros((P, 12), np.float32).tobytes()
    path.write_bytes(bytes(out))
    return path


def info_rc(path):
    cfg, P, K, fr = g.Config(), C.c_int(), C.c_int(), C.c_uint32()
    return g.lib().gmcs_checkpoint_info(bytes(str(path), "utf-8"), C.byref(cfg), C.byref(P), C.byref(K), C.byref(fr))


def test_layouts():
    assert C.sizeof(Header) == 232
    assert C.sizeof(TableHead) == 64


def test_well_formed_file_passes(tmp_path):
    p = write(tmp_path / "ok.ckpt", P=5, tables=((0, (4, 3, 2)), (0, (2, 2, 2))))
    cfg, P, K, fr = g.checkpoint_info(p)
    assert (P, K, fr) == (5, 2, 7) and cfg.k_nb == 3
    for dt in (1, 2):
        p = write(tmp_path / f"ok{dt}.ckpt", cfg=g.default_config(table_dtype=dt), tables=((dt, (5, 4, 3)),))
        assert g.checkpoint_info(p)[2] == 1
    p = write(tmp_path / "gicp.ckpt", cfg=g.default_config(model=g.MODEL_GICP), tables=((3, (2, 2, 1)),))
    assert g.checkpoint_info(p)[2] == 1
    p = write(tmp_path / "cols.ckpt", cfg=g.default_config(table_layout=g.LAYOUT_COLUMNS), tables=((0, (5, 4, 6)),))
    assert g.checkpoint_info(p)[2] == 1


@pytest.mark.parametrize("case", ["truncated", "extra_byte", "table_bytes", "table_dims", "huge_bytes",
                                  "dtype_vs_config", "unknown_dtype", "bad_config", "occ_bytes", "bad_grid_h",
                                  "version", "magic", "negative_K", "layout_vs_config", "cols_short_records",
                                  "cols_run_past_lattice", "cols_run_past_records"])
def test_corrupted_files_are_refused(tmp_path, case):
    p = tmp_path / f"{case}.ckpt"
    tweaks = {
        "table_bytes": lambda n, o: setattr(o, "bytes", o.bytes + 16) if n == "table" else None,
        "table_dims": lambda n, o: o.grid.n.__setitem__(0, 40) if n == "table" else None,
        "huge_bytes": lambda n, o: setattr(o, "bytes", 1 << 62) if n == "table" else None,
        "unknown_dtype": lambda n, o: setattr(o, "dtype", 9) if n == "table" else None,
        "bad_grid_h": lambda n, o: setattr(o.grid, "h", -0.2) if n == "table" else None,
        "occ_bytes": lambda n, o: o.n.__setitem__(2, 5) if n == "occ" else None,
        "version": lambda n, o: setattr(o, "version", 2) if n == "header" else None,
        "magic": lambda n, o: setattr(o, "magic", b"GMCSCKPX") if n == "header" else None,
        "negative_K": lambda n, o: setattr(o, "K", -1) if n == "header" else None,
    }
    if case in tweaks:
        write(p, tweak=tweaks[case])
    elif case == "dtype_vs_config":
        write(p, cfg=g.default_config(table_dtype=1), tables=((0, (4, 3, 2)),))
    elif case == "layout_vs_config":
        cfg = g.default_config(table_layout=g.LAYOUT_COLUMNS)
        write(p, cfg=cfg, tables=((0, (5, 4, 6)),), tweak=lambda n, o: setattr(o, "layout", 0) if n == "table" else None)
    elif case == "cols_short_records":
        cfg = g.default_config(table_layout=g.LAYOUT_COLUMNS)
        write(p, cfg=cfg, tables=((0, (5, 4, 6)),), tweak=lambda n, o: setattr(o, "bytes", o.bytes - 16) if n == "table" else None)
    elif case in ("cols_run_past_lattice", "cols_run_past_records"):
        cfg = g.default_config(table_layout=g.LAYOUT_COLUMNS)

        def bad_dir(n, o):
            if n == "dir":
                if case == "cols_run_past_lattice":
                    o[1] = 4 | (2 << 16)          # zlo 4 + 2 cells > 5 cells per column
                else:
                    o[2 * 11] = 10 ** 6           # a run starting past the last record
        write(p, cfg=cfg, tables=((0, (5, 4, 6)),), tweak=bad_dir)
    elif case == "bad_config":
        write(p, cfg=g.default_config(k_nb=g.MAX_NB + 1))
    else:
        write(p)
        data = p.read_bytes()
        p.write_bytes(data[:-1] if case == "truncated" else data + b"\0")
    assert info_rc(p) == g.E_IO
    with pytest.raises(g.GmcsError) as e:
        g.checkpoint_info(p)
    assert e.value.code == g.E_IO


def test_missing_file_and_null_path(tmp_path):
    assert info_rc(tmp_path / "absent.ckpt") == g.E_IO
    assert g.lib().gmcs_checkpoint_info(None, None, None, None, None) == g.E_INVALID
