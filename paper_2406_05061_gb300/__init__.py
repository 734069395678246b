"""GB300 (sm_103a) ProgOT hot path: Sinkhorn potentials, progressive entropic map,
coupling marginals and the ProgOT solve behind the C ABI of include/progot.h.

Importing the package loads nothing; ``paper_2406_05061_gb300.native`` loads
libprogot.so on first use and raises if it is missing (there is no CPU fallback)."""

__version__ = "0.1.0"

_NATIVE_NAMES = (
    "sinkhorn_potentials", "entropic_map_apply", "coupling_marginals", "progot_solve",
    "progot_schedule_alpha", "progot_mean_cost", "progot_schedule_eps", "Workspace",
    "workspace_size", "set_stall_window", "launch_count", "last_error", "ProgOTError",
)


def __getattr__(name):
    if name in _NATIVE_NAMES:
        from . import native
        return getattr(native, name)
    raise AttributeError(name)
