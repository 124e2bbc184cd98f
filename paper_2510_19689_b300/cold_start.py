"""Cold start of a fresh process: the serverless function's first call.

    python -m paper_2510_19689_b300.cold_start c1 [rows] [precision] [notorch]

Prints one JSON line with the milliseconds each stage of a cold start takes
in this process: PyTorch import and CUDA context creation, loading
libtabnet.so, `tabnet_create` (blob parse and validation, BN folding,
weight packing, upload and the launch-shape choice), the first forward of a
`rows`-row batch through host buffers (the first launch also loads the
kernel module), and a second, warm forward of the same batch.  With
`notorch` the process never imports PyTorch (the host-buffer call needs
only numpy), and the CUDA context is created inside `tabnet_create`.  The paper
quotes 2-5 s of model load and 1-2 s of CUDA initialisation for its GPU
functions (Sec. VI-B); this measures the same stages for this library.
"""
import json
import sys
import time

T_START = time.perf_counter()


def main(argv):
    name = argv[1] if len(argv) > 1 else "c1"
    rows = int(argv[2]) if len(argv) > 2 else 1000
    precision = argv[3] if len(argv) > 3 else "bf16x3"
    with_torch = not (len(argv) > 4 and argv[4] == "notorch")
    out = {"workload": name, "rows": rows, "precision": precision, "with_torch": with_torch}
    if with_torch:
        t = time.perf_counter()
        import torch
        torch.cuda.init()
        torch.zeros(1, device="cuda").item()
        out["torch_import_and_cuda_init_ms"] = (time.perf_counter() - t) * 1e3
    # without PyTorch the CUDA context is created inside tabnet_create
    t = time.perf_counter()
    from . import synth, tabnet
    out["package_import_ms"] = (time.perf_counter() - t) * 1e3
    t = time.perf_counter()
    _, blob, x_num, x_cat = synth.load_config(name, rows=rows)
    out["synthetic_inputs_ms"] = (time.perf_counter() - t) * 1e3
    t = time.perf_counter()
    tabnet.lib()
    out["library_load_ms"] = (time.perf_counter() - t) * 1e3
    t = time.perf_counter()
    m = tabnet.Model(blob, precision)
    out["create_ms"] = (time.perf_counter() - t) * 1e3
    for key in ("first_forward_ms", "warm_forward_ms"):
        t = time.perf_counter()
        m.forward_host(x_num, x_cat)
        out[key] = (time.perf_counter() - t) * 1e3
    out["status"] = m.poll_status()
    out["process_to_first_result_ms"] = (time.perf_counter() - T_START) * 1e3 - out["warm_forward_ms"]
    m.close()
    print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
