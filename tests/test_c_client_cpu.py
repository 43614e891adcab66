"""The boundary from C: a C11 program that includes include/ea_ageing.h compiles
with warnings as errors, links against the library, and gets from the host-only
calls (no GPU) the values the oracle gives."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as ora

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")

PROGRAM = r"""
#include <inttypes.h>
#include <stdio.h>
#include "ea_ageing.h"

int main(void)
{
    static const int sides[] = {2, 6, 16, 48, 128};
    for (unsigned i = 0; i < sizeof(sides) / sizeof(sides[0]); ++i) {
        int g[6];
        if (ea_geometry(sides[i], g) != EA_OK)
            return 2;
        printf("geometry %d %d %d %d %d %d %d\n", sides[i], g[0], g[1], g[2], g[3], g[4], g[5]);
    }
    int g[6];
    printf("odd %d %s\n", ea_geometry(7, g), ea_status_string(ea_geometry(7, g)));
    for (int rule = 0; rule < 2; ++rule) {
        uint64_t thr[7];
        uint8_t always[7];
        if (ea_thresholds(0.7, rule, thr, always) != EA_OK)
            return 3;
        printf("thresholds %d", rule);
        for (int k = 0; k < 7; ++k)
            printf(" %" PRIu64 ":%u", thr[k], (unsigned)always[k]);
        printf("\n");
    }
    uint64_t C[33];
    if (ea_geo_table(0.25, C) != EA_OK)
        return 4;
    printf("geo");
    for (int k = 0; k < 33; ++k)
        printf(" %" PRIu64, C[k]);
    printf("\n");
    int nb = 0;
    if (ea_c4_radial_bins(128, &nb) != EA_OK)
        return 5;
    printf("bins %d\n", nb);
    return 0;
}
"""


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc is not installed")
    from paper_1411_5512_gb300 import build, _lib
    build.build()
    libdir = os.path.dirname(_lib.LIB_PATH)
    d = tmp_path_factory.mktemp("c_client")
    src = d / "client.c"
    src.write_text(PROGRAM)
    exe = str(d / "client")
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic",
                           "-I", INCLUDE, str(src), "-o", exe, "-L", libdir, "-lea_gb300",
                           "-Wl,-rpath," + libdir])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    return out.stdout.splitlines()


def test_geometry_from_c(client):
    rows = [ln.split() for ln in client if ln.startswith("geometry ")]
    assert len(rows) == 5
    for row in rows:
        L = int(row[1])
        assert tuple(int(v) for v in row[2:]) == ora.geometry(L)
    odd = next(ln for ln in client if ln.startswith("odd ")).split()
    assert int(odd[1]) == -1 and "INVALID" in odd[2].upper()


def test_thresholds_and_gap_table_from_c(client):
    for rule in (0, 1):
        row = next(ln for ln in client if ln.startswith("thresholds %d " % rule)).split()[2:]
        thr, alw = ora.thresholds(0.7, rule)
        assert [int(v.split(":")[0]) for v in row] == [int(x) for x in thr]
        assert [int(v.split(":")[1]) for v in row] == [int(x) for x in alw]
    geo = [int(v) for v in next(ln for ln in client if ln.startswith("geo ")).split()[1:]]
    assert geo == [int(x) for x in ora.geo_table(0.25)]
    assert np.all(np.diff(np.array(geo, dtype=np.float64)) > 0)


def test_radial_bins_from_c(client):
    assert next(ln for ln in client if ln.startswith("bins ")).split()[1] == str(3 * 64 ** 2 + 1)
