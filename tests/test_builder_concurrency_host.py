"""Plans built concurrently on the native builder pool equal plans built one
at a time (CPU only, host-only plans).

The plan builder keeps per-thread scratch (spine levels, staging segments,
merge tables) and a per-thread rounding rule.  Builds of different
configurations (boundaries, split rules, both slope rounding rules, eager
adjoint tables, spine chunking) run on six pool threads at once, each
configuration three times, and every table of every plan must equal, byte
for byte, the same configuration built serially through fht_plan.
"""
import ctypes
import time

from paper_2411_07351_gb300 import _capi as C

CONFIGS = [
    # h, w, boundary, split, with_adjoint, rounding, spine_chunk
    (300, 500, C.FHT_CYCLIC, C.FHT_SPLIT_T, 0, 0, 0),
    (300, 500, C.FHT_CYCLIC, C.FHT_SPLIT_T, 0, 1, 0),
    (1000, 257, C.FHT_EXTENDED, C.FHT_SPLIT_T, 1, 0, 0),
    (1000, 257, C.FHT_EXTENDED, C.FHT_SPLIT_T, 1, 1, 2),
    (2100, 333, C.FHT_CYCLIC, C.FHT_SPLIT_T, 0, 0, 1),
    (777, 1500, C.FHT_EXTENDED, C.FHT_SPLIT_S, 1, 0, 0),
    (131, 45, C.FHT_CYCLIC, C.FHT_SPLIT_S, 0, 1, 0),
    (4097, 90, C.FHT_EXTENDED, C.FHT_SPLIT_T, 0, 0, 0),
]


def _tuning(adj, rounding, chunk):
    return C.fht_tuning_t(0, 0, 0, int(adj), int(rounding), int(chunk), 0)


def _tables(lib, h):
    out = []
    for k in range(14):
        data, count, esz = ctypes.c_void_p(), ctypes.c_int64(), ctypes.c_int32()
        C.check(lib.fht_plan_table(h, k, ctypes.byref(data), ctypes.byref(count), ctypes.byref(esz)),
                "fht_plan_table")
        n = count.value * esz.value
        out.append(ctypes.string_at(data.value, n) if n else b"")
    return out


def test_pool_builds_equal_serial_builds():
    lib = C.load()
    serial = {}
    for cfg in CONFIGS:
        h, w, b, s, adj, rnd, ch = cfg
        p = ctypes.c_void_p()
        tun = _tuning(adj, rnd, ch)
        C.check(lib.fht_plan(ctypes.byref(p), h, w, C.FHT_U8_I32, C.FHT_QALL, b, s, -1, ctypes.byref(tun)), "fht_plan")
        serial[cfg] = _tables(lib, p)
        lib.fht_plan_destroy(p)

    pool = ctypes.c_void_p()
    C.check(lib.fht_builder_create(ctypes.byref(pool), 6), "fht_builder_create")
    try:
        want = {}
        tag = 0
        for rep in range(3):
            for cfg in CONFIGS:
                h, w, b, s, adj, rnd, ch = cfg
                tun = _tuning(adj, rnd, ch)
                C.check(lib.fht_builder_submit(pool, tag, h, w, C.FHT_U8_I32, C.FHT_QALL, b, s, -1, ctypes.byref(tun)),
                        "fht_builder_submit")
                want[tag] = cfg
                tag += 1
        cap = 64
        tags = (ctypes.c_uint64 * cap)()
        plans = (ctypes.c_void_p * cap)()
        status = (ctypes.c_int * cap)()
        n = ctypes.c_int32()
        done, deadline = 0, time.time() + 120
        while done < len(want) and time.time() < deadline:
            C.check(lib.fht_builder_poll(pool, tags, plans, status, cap, ctypes.byref(n)), "fht_builder_poll")
            for k in range(n.value):
                cfg = want[int(tags[k])]
                assert status[k] == C.FHT_OK, cfg
                got = _tables(lib, ctypes.c_void_p(plans[k]))
                lib.fht_plan_destroy(ctypes.c_void_p(plans[k]))
                for t, (a, e) in enumerate(zip(got, serial[cfg])):
                    assert a == e, f"table {t} of {cfg} differs when built on the pool"
                done += 1
            if n.value == 0:
                time.sleep(0.005)
        assert done == len(want)
    finally:
        lib.fht_builder_destroy(pool)
