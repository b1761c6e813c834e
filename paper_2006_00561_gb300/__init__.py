"""GB300 population-annealing engine (C ABI in include/pa.h, kernels in csrc/)."""
from .pa import (  # noqa: F401
    Config, Obs, PaError, Run, make_config, pa_dump, pa_dump_range, pa_free, pa_init, pa_num_bins,
    pa_observables, pa_observables_history, pa_resample, pa_run_steps, pa_status, pa_step,
    pa_sweep, pa_tables, pa_workspace_size,
)
