"""A minimal NVTX tool for the tests: a shared library that attaches
through NVTX's injection interface (NVTX_INJECTION64_PATH) and writes every
range push and pop of the process to the file named by NVTX_RECORD."""
import os
import subprocess

INJECTION_C = r"""
#include <stdio.h>
#include <stdlib.h>
#include <nvtx3/nvToolsExt.h>

static FILE* out;

static int push_a(const char* name) {
    fprintf(out, "push %s\n", name);
    fflush(out);
    return 0;
}

static int pop(void) {
    fprintf(out, "pop\n");
    fflush(out);
    return 0;
}

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table) {
    const NvtxExportTableCallbacks* cb = (const NvtxExportTableCallbacks*)get_table(NVTX_ETID_CALLBACKS);
    NvtxFunctionTable table = 0;
    unsigned int size = 0;
    if (!cb || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &size)) return 0;
    if (size <= NVTX_CBID_CORE_RangePop) return 0;
    out = fopen(getenv("NVTX_RECORD"), "w");
    if (!out) return 0;
    *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)push_a;
    *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)pop;
    return 1;
}
"""


def compile_tool(directory):
    """Builds the tool in `directory`; returns the library's path."""
    from paper_2607_00756_gb300 import build
    src = os.path.join(directory, "nvtx_record.c")
    so = os.path.join(directory, "libnvtx_record.so")
    with open(src, "w") as f:
        f.write(INJECTION_C)
    inc = os.path.join(build._cuda_home(), "include")
    r = subprocess.run(["gcc", "-shared", "-fPIC", "-O1", "-I", inc, src, "-o", so], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(r.stderr)
    return so


def nesting_ok(lines):
    """True if every pop closes an open push and none stays open."""
    depth = 0
    for ln in lines:
        depth += 1 if ln.startswith("push ") else -1
        if depth < 0:
            return False
    return depth == 0
