"""Element constants used as inputs.

Atomic numbers and standard atomic masses are IUPAC values.  Surface binding
energies U_s are the cohesive energies commonly used for sputtering (the paper
lets SIMTRA choose U_s per element, Sec. "The calculations were performed with
pySIMTRA"; the Ni value 4.44 eV is the one the quaternary workload fixes).
Bulk densities (g/cm^3) are used only when arrival fractions are converted to
atomic percent (the density / atomic-mass weighting described after Table 1).
"""

from dataclasses import dataclass


@dataclass(frozen=True)
class Element:
    symbol: str
    Z: int
    mass: float      # u
    U_s: float       # eV, surface binding energy
    density: float   # g/cm^3, nominal bulk density


ELEMENTS = {
    "Ni": Element("Ni", 28, 58.6934, 4.44, 8.908),
    "Pd": Element("Pd", 46, 106.42, 3.89, 12.023),
    "Pt": Element("Pt", 78, 195.084, 5.84, 21.45),
    "Ru": Element("Ru", 44, 101.07, 6.74, 12.45),
    "Cu": Element("Cu", 29, 63.546, 3.49, 8.96),
    "Ti": Element("Ti", 22, 47.867, 4.85, 4.506),
}

GAS_AR = Element("Ar", 18, 39.948, 0.0, 0.0)


def element(symbol: str) -> Element:
    return ELEMENTS[symbol]
