"""GB300-native parallel acceptance-rejection selection of the next reaction
for the Stochastic Simulation Algorithm (Neri & Mestivier, 2014).

* ``binding``   -- Python mirror of the C ABI in include/gbar.h (libgbar.so).
* ``build``     -- compiles libgbar.so for sm_103a with nvcc.
* ``workloads`` -- seeded synthetic inputs (no method arithmetic).

The binding module is imported lazily so that the input generators can be
used without a GPU; any selection call without the built library raises.
"""
__all__ = ["binding", "build", "workloads"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
