"""Run the batched forward pass on one synthetic workload (for profilers).

    python -m paper_2510_19689_b300.run_workload c2 bf16x3 [rows] [nwg,slots,ctas_per_sm | -] [launches]

Builds the named workload's seeded model and rows (synth.load_config), moves
the rows to cuda:0, optionally fixes the launch shape, runs `launches`
forward calls (default 4) through the C ABI and prints the status word.
It is the command the kernel summaries under profiles/ were captured with:
the launches are the library's own, nothing else runs on the device.
"""
import sys

import torch

from . import synth, tabnet


def main(argv):
    name = argv[1] if len(argv) > 1 else "c2"
    precision = argv[2] if len(argv) > 2 else "bf16x3"
    rows = int(argv[3]) if len(argv) > 3 else synth.ROWS[name]
    shape = tuple(int(v) for v in argv[4].split(",")) if len(argv) > 4 and argv[4] != "-" else None
    launches = int(argv[5]) if len(argv) > 5 else 4
    _, blob, x_num, x_cat = synth.load_config(name, rows=rows)
    m = tabnet.Model(blob, precision)
    if shape is not None:
        m.set_tile_config(*shape)
    dev = torch.device("cuda", 0)
    xn = torch.from_numpy(x_num).to(dev)
    xc = torch.from_numpy(x_cat).to(dev)
    logits, masks, agg = m.run(xn, xc)
    for _ in range(launches - 1):
        m.forward(xn, xc, rows, logits, masks, agg)
    torch.cuda.synchronize()
    status = m.poll_status()
    shape_s = m.tile_config() if precision != "fp32" else "cuda cores"
    print(f"{name} {precision} rows={rows} shape={shape_s} launches={launches} status={status}")
    m.close()
    return 0 if status == 0 else 1


if __name__ == "__main__":
    sys.exit(main(sys.argv))
